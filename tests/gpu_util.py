"""Helpers for the GPU tests: run the CUDA path through the C ABI."""

import numpy as np

import paper_1705_02043_gb300 as pk


def run(kernel, periodic, src, dens, trg, p=6, leaf=32, depth=10, precision=0, ell=2,
        lo=(0.0, 0.0, 0.0), L=1.0, cache_dir=None, return_plan=False, precompute="device"):
    """Evaluate on cuda:0; dens [S] / [S,3] / [nrhs,S,k]; returns numpy [nrhs?,T,k?]."""
    import torch
    k = 1 if kernel == 0 else 3
    d = np.asarray(dens, dtype=np.float64)
    squeeze = d.ndim == (1 if k == 1 else 2)
    d = d.reshape(-1, len(src), k)
    nrhs = d.shape[0]
    plan = pk.PeriodicKIFMM(kernel, periodic, lo, L, p, ell, leaf, depth, precision, nrhs, cache_dir,
                            precompute=precompute)
    dev = torch.device("cuda:0")
    ts = torch.tensor(np.asarray(src, np.float64), device=dev).contiguous()
    td = torch.tensor(d, device=dev).contiguous()
    tt = torch.tensor(np.asarray(trg, np.float64), device=dev).contiguous()
    out = plan.evaluate(ts, td, tt)
    torch.cuda.synchronize()
    out = out.cpu().numpy()
    if squeeze:
        out = out[0, :, 0] if k == 1 else out[0]
    if return_plan:
        return out, plan
    plan.close()
    return out


def rel_l2(u, ref):
    u, ref = np.asarray(u).ravel(), np.asarray(ref).ravel()
    return float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
