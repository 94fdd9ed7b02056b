"""Shared helpers of the GPU parity tests: run a workload through the C ABI
and through the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

from oracle.rte import Solver


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_forward(wl, ckpt=0, snaps=None, groups=None, precision=0, flags=0):
    from paper_2202_09421_gb300.solver import FCDOMSolver
    dev = torch.device("cuda:0")
    a = torch.tensor(wl.mua, dtype=torch.float32, device=dev)
    b = torch.tensor(wl.mus, dtype=torch.float32, device=dev)
    s = FCDOMSolver(wl.grid, wl.optics, a, b, wl.c, wl.dt, ckpt_interval=ckpt, precision=precision,
                    flags=flags)
    groups = wl.groups if groups is None else groups
    snaps = list(wl.snap_steps) if snaps is None else snaps
    fl = s.forward(groups, wl.n_steps, snaps)
    curves = s.readout(wl.detectors)
    torch.cuda.synchronize()
    return s, (fl.cpu().numpy() if fl is not None else None), curves.cpu().numpy()


def oracle_forward(wl, groups=None, snaps=None, keep_u=False):
    S = Solver(wl)
    groups = wl.groups if groups is None else groups
    snaps = list(wl.snap_steps) if snaps is None else snaps
    curves, fl, us = [], [], []
    for g in groups:
        out = S.forward(g, wl.n_steps, wl.detectors, snap_steps=snaps)
        curves.append(out["curves"])
        fl.append([out["fluence"][k] for k in snaps])
        us.append(out["u"])
    return np.array(curves), np.array(fl), us
