"""Shared helpers for the GPU parity tests: run the CUDA path through the C ABI."""
import numpy as np
import torch

from paper_2103_08513_gb300 import MRCM


def gpu_solver(w, precision="fp64", bc_type=((0, 0),) * 3, bc_value=((0.0, 0.0),) * 3,
               ir_max_sweeps=6, ir_tol=1e-14, interface_refine=0, fallback_cap=0):
    return MRCM(w.n, w.edges, w.patch, h=w.h, beta_mode=w.beta_mode, alpha=w.alpha,
                beta_const=w.beta_const, bc_type=bc_type, bc_value=bc_value, precision=precision,
                ir_max_sweeps=ir_max_sweeps, ir_tol=ir_tol, interface_refine=interface_refine,
                fallback_cap=fallback_cap)


def run_gpu(w, K, f, precision="fp64", **kw):
    s = gpu_solver(w, precision, **kw)
    Kd = torch.from_numpy(np.ascontiguousarray(K)).cuda()
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    p, u, X, mres = s.solve(Kd, fd)
    torch.cuda.synchronize()
    code, st = s.read_status()
    return s, p.cpu().numpy().ravel(), u.cpu().numpy(), X.cpu().numpy(), float(mres.cpu()[0]), code, st


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
