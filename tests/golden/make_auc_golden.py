"""Writes auc_rmat20_20epochs.json: the FP64 oracle's held-out link-prediction
AUC and loss after 20 epochs of the benchmark workload.

Workload: R-MAT scale 20 (16 * 2^20 directed edges, a = .57, b = c = .19),
symmetrised, 5% of the undirected edges held out (graphs.rmat_holdout_graph),
d = 128, s = 5, minibatch 4096, eta_0 = 0.02 decayed linearly over 20 epochs,
seed 1; Algorithm 1 with the per-pair gradients of Eq. 8/9 (t model) and
Eq. 5/6 (sigmoid model), as the oracle computes them.  The AUC scores a pair
by -|z_u - z_v|^2 (t) or z_u . z_v (sigmoid) and counts ties as one half; the
loss is Eq. 2 (with Eq. 7 or Eq. 3) over the training graph, with the
negative samples of epoch 20.

Only oracle/ computes the values (FP64, no fused multiply-add, the same bits
for any thread count).  bench.py reports them beside the GPU's AUC, and the
GPU test of the 20-epoch AUC checks them against the oracle run live.

    python tests/golden/make_auc_golden.py      # a few minutes of CPU
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2009_10035_gb300 import graphs  # noqa: E402

OUT = os.path.join(HERE, "auc_rmat20_20epochs.json")


def main():
    g = graphs.rmat_holdout_graph()
    d, s, b, lr, epochs, seed = 128, 5, 4096, 0.02, 20, 1
    out = {
        "_about": ("FP64 oracle after 20 epochs of Algorithm 1 on R-MAT scale 20 with 5% of "
                   "the undirected edges held out (d 128, s 5, minibatch 4096, eta 0.02 "
                   "decayed linearly over 20 epochs, seed 1): held-out link-prediction AUC "
                   "and the loss of Eq. 2 with the negative samples of epoch 20.  Written by "
                   "tests/golden/make_auc_golden.py, which calls only oracle/."),
        "graph": {"n": int(g.n), "nnz": int(g.nnz), "test_pos": int(g.test_pos.shape[0]),
                  "test_neg": int(g.test_neg.shape[0])},
        "models": {},
    }
    for name, model in (("tdist", oracle.TDIST), ("sigmoid", oracle.SIGMOID)):
        t0 = time.perf_counter()
        Z = oracle.train(model, g.row_ptr, g.col_idx, oracle.init_embedding(g.n, d, seed), s, b,
                         seed, lr, epochs, schedule=1, total_epochs=epochs)
        auc = oracle.link_auc(model, Z, g.test_pos, g.test_neg)
        loss = oracle.loss_total(model, g.row_ptr, g.col_idx, Z, s, seed, epochs)
        out["models"][name] = {"auc": auc, "loss": loss}
        print(f"{name}: auc {auc:.6f} loss {loss:.6e} ({time.perf_counter() - t0:.0f} s)",
              flush=True)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
