"""Writes or_rbm_params.txt: OR-gate clause-RBM parameter sets fitted and
quantised by the CPU oracle only (Sec. 4.1 "Learning OR gate RBM parameters";
appendix "Pretraining": Adam, learning rate 1e-3, 3 hidden units for K = 3 and
K + 1 above). Targets F* in {0.068, 0.528} are the paper's 1-TPU condition
(appendix "Pretraining"); weight bucket j uses F* (1 + 0.5 j).

    python tests/golden/make_rbm_params.py
"""
import os
import sys

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))
import oracle  # noqa: E402

FSTARS = [0.068, 0.528]
BUCKETS = 4
GAMMA = 0.5
Q = 4

if __name__ == "__main__":
    table = oracle.make_table(range(1, 13), FSTARS, n_buckets=BUCKETS, gamma=GAMMA, Q=Q)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "or_rbm_params.txt")
    table.save(out, header=(
        "OR-gate clause RBMs fitted by oracle.fit_or_rbm and quantised by oracle.quantise\n"
        f"(W on the 2^-{Q} grid, b on the 2^-24 grid). Keys: length, weight bucket, temperature.\n"
        f"Temperatures: F* = {FSTARS} (appendix 'Pretraining', 1-TPU condition);\n"
        f"bucket j target = F* (1 + {GAMMA} j). Written by tests/golden/make_rbm_params.py."))
    print("wrote", out, len(table.sets), "sets")
