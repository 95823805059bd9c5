"""Training pipeline of the active-block predictor (rac_predictor_* and
rac_enforce_learned in include/rac.h).

  collect_traces(items)   run the Proposition-2 recurrence on the GPU with
                          trace records on, for a list of (network, states)
                          items; returns the features and labels of every
                          candidate (slab, state) pair, still on the device;
  train(x, y, ...)        a new Predictor trained by the library's kernels;
  choose_threshold(...)   the logit threshold that keeps a given fraction of
                          the positive training samples (logits from the
                          tensor-core routine the sweep kernel runs).

Host code only orchestrates: every sweep, feature, label, gradient and
logit comes from the library's kernels.
"""
import numpy as np

from . import (PREDICTOR_FEATURES, Predictor, Trace, enforce_learned)


def _torch():
    import torch
    return torch


def collect_traces(items, stream=None):
    """items: iterable of (Network, states) with states a (B, n) uint32
    CUDA tensor.  Returns (x, y, info): x (N, 8) and y (N,) float32 CUDA
    tensors, info a list of per-item dicts (records, evaluations, sweeps)."""
    torch = _torch()
    xs, ys, info = [], [], []
    for net, states in items:
        B = states.shape[0]
        slabs = net.info()["n_slabs"]
        cap = slabs * B * 8
        while True:
            trace = Trace(cap)
            out = torch.empty_like(states)
            sweeps = torch.empty(B, dtype=torch.int32, device=states.device)
            status = torch.empty(B, dtype=torch.int32, device=states.device)
            enforce_learned(net, states, out, sweeps, status, predictor=None, trace=trace,
                            stream=stream)
            torch.cuda.synchronize()
            count = trace.count()
            if count <= cap:
                break
            cap = count
        xs.append(trace.features[:count].clone())
        ys.append(trace.label[:count].clone())
        info.append({"records": count, "evaluated": trace.evaluated(),
                     "sweeps": sweeps.cpu().numpy()})
    x = torch.cat(xs) if xs else torch.empty((0, PREDICTOR_FEATURES), device="cuda")
    y = torch.cat(ys) if ys else torch.empty(0, device="cuda")
    return x, y, info


def train(x, y, steps=3000, batch=4096, lr=2e-3, pos_weight=4.0, seed=0, init_seed=0):
    """A predictor trained on (x, y) with Adam on the GPU."""
    pred = Predictor(init_seed)
    pred.train(x, y, steps=steps, batch=batch, lr=lr, pos_weight=pos_weight, seed=seed)
    return pred


def logits(pred, x):
    torch = _torch()
    z = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    pred.predict(x, z, tensor_cores=True)
    return z


def choose_threshold(pred, x, y, recall=0.98):
    """Largest logit threshold that still keeps `recall` of the positives."""
    z = logits(pred, x).cpu().numpy()
    pos = np.sort(z[y.cpu().numpy() > 0.5])
    if pos.shape[0] == 0:
        return 0.0
    i = int(np.floor((1.0 - recall) * pos.shape[0]))
    # evaluated iff logit > threshold: step just below the chosen positive
    return float(np.nextafter(np.float32(pos[i]), np.float32(-np.inf)))
