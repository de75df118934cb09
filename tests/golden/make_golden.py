"""Writes the stored expected values under tests/golden/ that are computed, not
printed in the paper.  Calls only the oracle."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

if __name__ == "__main__":
    g = {"cite": "Sec. 5.2 GMRF on a square grid; exact value from the separable Dirichlet-Laplacian spectrum",
         "N": 1000, "kappa2": 0.1, "logdet": oracle.grid_laplacian_logdet(1000, 0.1),
         "written_by": "tests/golden/make_golden.py (oracle.grid_laplacian_logdet)"}
    json.dump(g, open(os.path.join(HERE, "grid_gmrf_logdet.json"), "w"), indent=2)
    print(g)
