"""Training the learned frontier's predictor on the engine's own traces.

`train_for` normalises a copy of the workload in frontier mode while sampling
training rows (trs_collect_samples: features of nodes not in normal form every
`period` sweeps, labelled by whether they act within the next `period`
sweeps), then trains the predictor on the GPU with its own forward/backward
and Adam kernels (trs_predictor_train).
"""
from __future__ import annotations

import paper_2009_07174_gb300 as trs


def train_for(program, flat, offs, capacity: int, period: int = 16, rate: float = 1.0,
              max_rows: int = 1 << 21, epochs: int = 8, lr: float = 5e-3, seed: int = 1,
              return_info: bool = False):
    pool = trs.Pool(program, capacity)
    pool.term_upload_batch(flat, offs)
    samples = trs.Samples(program, max_rows)
    n, st = pool.trs_collect_samples(samples, period=period, rate=rate, seed=seed, mode="frontier")
    del pool
    pred = trs.Predictor(program, seed=seed)
    losses = pred.train(samples, n, epochs=epochs, batch=4096, lr=lr)
    if return_info:
        return pred, {"rows": n, "losses": [float(x) for x in losses],
                      "positive_rate": float(samples.label[:n].mean().item())}
    return pred
