"""Writes exact_ising.json: exact e = -<E>/N and C_V = beta^2 var(E)/N of the
periodic L x L Ising ferromagnet (the closed form of oracle/ising_exact.py,
Kaufman / Ferdinand-Fisher) for the lattices the statistical GPU tests use.
Run from the repository root:  python tests/golden/make_exact_ising.py
"""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ising_exact as X  # noqa: E402

BETA_C = math.log(1 + math.sqrt(2)) / 2
CASES = [(16, 0.4), (32, 0.4), (64, 0.4), (64, BETA_C), (128, 0.4), (1024, 0.4), (1024, BETA_C)]

out = {"_source": "oracle/ising_exact.py (Kaufman 1949, Ferdinand-Fisher 1969 closed form), 40 digits",
       "cases": []}
for L, beta in CASES:
    e, cv = X.exact_e_cv(L, beta)
    out["cases"].append({"L": L, "beta": beta, "e": e, "C_V": cv})
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "exact_ising.json"), "w") as f:
    json.dump(out, f, indent=1)
print(json.dumps(out, indent=1))
