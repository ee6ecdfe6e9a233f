"""Python binding of libmrcm: argument marshalling around the C ABI.

PyTorch provides device memory and streams; every step of the solve runs in
the library's CUDA kernels.  Method names match the C entry points
(include/mrcm.h) without the ``mrcm_`` prefix.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class MRCM:
    """One MRCM problem (grid, decomposition, interface space) bound to one GPU.

    Parameters follow the mrcm_config struct: ``n = (nx, ny, nz)``,
    ``h = (hx, hy, hz)``, ``edges`` = per-axis subdomain edge lists,
    ``patch = ((p1, p2) for x-, y-, z-normal faces)`` (0 = whole face).
    """

    def __init__(self, n, edges, patch=((0, 0),) * 3, h=(1.0, 1.0, 1.0), beta_mode=0, alpha=1.0,
                 beta_const=1.0, bc_type=((0, 0),) * 3, bc_value=((0.0, 0.0),) * 3,
                 precision="fp64", ir_max_sweeps=4, ir_tol=1e-14, device=None, allocate=True, tune_cache=None,
                 wave_bytes=0, interface_refine=0, fallback_cap=0):
        self.lib = L.load()
        cfg = L.mrcm_config()
        cfg.nx, cfg.ny, cfg.nz = (int(v) for v in n)
        cfg.hx, cfg.hy, cfg.hz = (float(v) for v in h)
        self._cuts = []
        for a in range(3):
            arr = (C.c_int * len(edges[a]))(*[int(e) for e in edges[a]])
            self._cuts.append(arr)
            cfg.n_cuts[a] = len(edges[a])
            cfg.cuts[a] = C.cast(arr, C.POINTER(C.c_int))
            cfg.patch[a][0], cfg.patch[a][1] = int(patch[a][0]), int(patch[a][1])
            cfg.bc_type[a][0], cfg.bc_type[a][1] = int(bc_type[a][0]), int(bc_type[a][1])
            cfg.bc_value[a][0], cfg.bc_value[a][1] = float(bc_value[a][0]), float(bc_value[a][1])
        cfg.beta_mode = int(beta_mode)
        cfg.alpha = float(alpha)
        cfg.beta_const = float(beta_const)
        cfg.precision = L.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg.ir_max_sweeps = int(ir_max_sweeps)
        cfg.ir_tol = float(ir_tol)
        cfg.wave_bytes = int(wave_bytes)
        cfg.interface_refine = int(interface_refine)
        cfg.fallback_cap = int(fallback_cap)
        self._tune_cache = tune_cache.encode() if tune_cache else None
        cfg.tune_cache = self._tune_cache
        self.cfg = cfg
        self.n = tuple(int(v) for v in n)
        h_ = C.c_void_p()
        L.check(self.lib.mrcm_setup(C.byref(cfg), C.byref(h_)))
        self.handle = h_
        wsb, nif = C.c_size_t(), C.c_size_t()
        L.check(self.lib.mrcm_query_workspace(self.handle, C.byref(wsb), C.byref(nif)), self.handle)
        self.ws_bytes = int(wsb.value)
        self.n_interface = int(nif.value)
        sz = L.mrcm_sizes()
        L.check(self.lib.mrcm_query_sizes(self.handle, C.byref(sz)), self.handle)
        self.sizes = {k: getattr(sz, k) for k, _ in L.mrcm_sizes._fields_}
        self.device = torch.device(device if device is not None else "cuda")
        self.ws = None
        if allocate:
            self.allocate()

    # ------------------------------------------------------------------ memory
    def allocate(self):
        """Allocate the workspace (caller-owned device memory, 256-byte aligned)."""
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self._ws_off = (-base) % 256
        return self.ws

    @property
    def ws_ptr(self):
        return C.c_void_p(self.ws.data_ptr() + self._ws_off)

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                self.lib.mrcm_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    # ------------------------------------------------------------------ steps
    def factor_local(self, K, stream=None):
        assert K.dtype == torch.float64 and K.is_cuda and K.is_contiguous()
        self._K = K
        L.check(self.lib.mrcm_factor_local(self.handle, _ptr(K), self.ws_ptr, C.c_size_t(self.ws_bytes),
                                           _stream(stream)), self.handle)

    def solve_mbf(self, f, stream=None):
        assert f.dtype == torch.float64 and f.is_cuda and f.is_contiguous()
        self._f = f
        L.check(self.lib.mrcm_solve_mbf(self.handle, _ptr(f), self.ws_ptr, _stream(stream)), self.handle)

    def solve_mbf_learned(self, f, net=None, pred=None, cg_maxit=200, max_outer=8, stream=None):
        """Learned-form MBFs (precision "learned_pcg"): warm-started FP32 CG inside FP64
        refinement, FP64 direct fallback; pred = the network's P-MBF predictions in
        sample order (or None: from zero)."""
        assert f.dtype == torch.float64 and f.is_cuda and f.is_contiguous()
        self._f = f
        n_pred = int(pred.shape[0]) if pred is not None else 0
        L.check(self.lib.mrcm_solve_mbf_learned(self.handle, net.net if net is not None else None,
                                                _ptr(pred) if pred is not None else None, n_pred, _ptr(f),
                                                int(cg_maxit), int(max_outer), self.ws_ptr, _stream(stream)),
                self.handle)

    def read_cg_iterations(self):
        v = C.c_longlong()
        L.check(self.lib.mrcm_read_cg_iterations(self.handle, self.ws_ptr, C.byref(v)), self.handle)
        return int(v.value)

    def assemble_interface(self, stream=None):
        L.check(self.lib.mrcm_assemble_interface(self.handle, self.ws_ptr, _stream(stream)), self.handle)

    def solve_interface(self, X=None, stream=None):
        if X is None:
            X = torch.empty(max(self.n_interface, 1), dtype=torch.float64, device=self.device)
        L.check(self.lib.mrcm_solve_interface(self.handle, _ptr(X), self.ws_ptr, _stream(stream)), self.handle)
        return X

    def reconstruct(self, X, p=None, u=None, mres=None, stream=None):
        nx, ny, nz = self.n
        if p is None:
            p = torch.empty((nz, ny, nx), dtype=torch.float64, device=self.device)
        if u is None:
            u = torch.empty((6, nz, ny, nx), dtype=torch.float64, device=self.device)
        if mres is None:
            mres = torch.empty(1, dtype=torch.float64, device=self.device)
        L.check(self.lib.mrcm_reconstruct(self.handle, _ptr(X), _ptr(p), _ptr(u), _ptr(mres), self.ws_ptr,
                                          _stream(stream)), self.handle)
        return p, u, mres

    def postprocess_velocity(self, u, out=None, mres=None, stream=None):
        """Mean velocity post-processing of a reconstructed velocity u (6, nz, ny, nx);
        returns (u_pp, mass_residual_max).  Overwrites the local factors: the next
        solve starts again from factor_local."""
        assert u.dtype == torch.float64 and u.is_cuda and u.is_contiguous()
        if out is None:
            out = torch.empty_like(u)
        if mres is None:
            mres = torch.empty(1, dtype=torch.float64, device=self.device)
        L.check(self.lib.mrcm_postprocess_velocity(self.handle, _ptr(u), _ptr(out), _ptr(mres), self.ws_ptr,
                                                   _stream(stream)), self.handle)
        return out, mres

    def impes(self, K, f, S, mu_w=1.0, mu_o=5.0, cfl=0.9, C_skip=10, n_steps=10, stream=None):
        """Two-phase IMPES (Alg. overview-code): S (nz, ny, nx) is advanced in place by
        n_steps transport steps, with the MRCM solve + post-processing every C_skip
        steps; returns the simulated time (device tensor of one element)."""
        assert S.dtype == torch.float64 and S.is_cuda and S.is_contiguous()
        nb = C.c_size_t()
        L.check(self.lib.mrcm_transport_query(self.handle, C.byref(nb)), self.handle)
        if getattr(self, "_tws", None) is None or self._tws.numel() < nb.value:
            self._tws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        t = torch.zeros(1, dtype=torch.float64, device=self.device)
        L.check(self.lib.mrcm_impes(self.handle, _ptr(K), _ptr(f), _ptr(S), C.c_double(mu_w), C.c_double(mu_o),
                                    C.c_double(cfl), int(C_skip), int(n_steps), _ptr(t), _ptr(self._tws),
                                    C.c_size_t(self._tws.numel()), self.ws_ptr, C.c_size_t(self.ws_bytes),
                                    _stream(stream)), self.handle)
        return t

    def outputs(self):
        """Preallocated (X, p, u, mres) device buffers for solve(..., out=...)."""
        nx, ny, nz = self.n
        return (torch.empty(max(self.n_interface, 1), dtype=torch.float64, device=self.device),
                torch.empty((nz, ny, nx), dtype=torch.float64, device=self.device),
                torch.empty((6, nz, ny, nx), dtype=torch.float64, device=self.device),
                torch.empty(1, dtype=torch.float64, device=self.device))

    def solve(self, K, f, out=None, stream=None, graph=False):
        """All five device steps of one MRCM pressure solve; returns (p, u, X, mres).

        graph=True runs mrcm_solve in CUDA-graph mode (captured on the first call,
        replayed afterwards); it needs a non-default stream.
        """
        if graph:
            assert K.is_contiguous() and f.is_contiguous()
            X, p, u, mres = out if out is not None else self.outputs()
            self._K, self._f = K, f
            L.check(self.lib.mrcm_solve(self.handle, _ptr(K), _ptr(f), _ptr(X), _ptr(p), _ptr(u), _ptr(mres),
                                        self.ws_ptr, C.c_size_t(self.ws_bytes), _stream(stream), 1), self.handle)
            return p, u, X, mres
        self.factor_local(K, stream)
        self.solve_mbf(f, stream)
        self.assemble_interface(stream)
        if out is None:
            X = self.solve_interface(stream=stream)
            p, u, mres = self.reconstruct(X, stream=stream)
        else:
            X, p, u, mres = out
            self.solve_interface(X, stream=stream)
            self.reconstruct(X, p, u, mres, stream=stream)
        return p, u, X, mres

    def solve_host(self, K, f, X, p, u, mres=None, stream=None, graph=False):
        """mrcm_solve with host (CPU) tensors: K, f in; X, p, u (and mres) out, written
        once `stream` completes.  graph=True needs page-locked tensors."""
        for t in (K, f, X, p, u) + ((mres,) if mres is not None else ()):
            assert not t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
        L.check(self.lib.mrcm_solve_host(self.handle, _ptr(K), _ptr(f), _ptr(X), _ptr(p), _ptr(u),
                                         _ptr(mres) if mres is not None else None, self.ws_ptr,
                                         C.c_size_t(self.ws_bytes), _stream(stream), 1 if graph else 0), self.handle)
        return p, u, X, mres

    def tuning(self):
        """{'solve', 'sweep', 'factor_small', 'factor_mid'}: the kernel variants in use."""
        v = [C.c_int() for _ in range(4)]
        L.check(self.lib.mrcm_query_tuning(self.handle, *[C.byref(x) for x in v]), self.handle)
        return dict(zip(("solve", "sweep", "factor_small", "factor_mid"), (x.value for x in v)))

    def tuning_times(self):
        """{'first_solve', 'sweeps'}: per-variant median times (ms) of the last autotune (-1 = not
        timed), {'first_solve_ctas', 'sweeps_ctas'}: resident CTAs per SM of each variant."""
        cap = 16
        a, b = (C.c_float * cap)(), (C.c_float * cap)()
        oa, ob, n = (C.c_int * cap)(), (C.c_int * cap)(), C.c_int()
        sep, sep_ms = C.c_int(), C.c_float()
        L.check(self.lib.mrcm_read_tuning_times(self.handle, a, b, oa, ob, cap, C.byref(n), C.byref(sep),
                                                C.byref(sep_ms)), self.handle)
        k = min(cap, n.value)
        return {"first_solve": [round(float(a[i]), 4) for i in range(k)],
                "sweeps": [round(float(b[i]), 4) for i in range(k)],
                "first_solve_ctas": [int(oa[i]) for i in range(k)], "sweeps_ctas": [int(ob[i]) for i in range(k)],
                "sweeps_one_launch_each": bool(sep.value), "sweeps_one_launch_each_ms": round(float(sep_ms.value), 4)}

    def autotune(self, f, stream=None):
        """Pick the fastest local-solve kernel variants for this problem (after factor_local)."""
        v0, v1 = C.c_int(), C.c_int()
        L.check(self.lib.mrcm_autotune(self.handle, _ptr(f), self.ws_ptr, _stream(stream), C.byref(v0),
                                       C.byref(v1)), self.handle)
        return int(v0.value), int(v1.value)

    # ------------------------------------------------------------------ profiling
    def profile(self, enable=True):
        """Start (or stop) per-kernel CUDA-event timing inside the library."""
        L.check(self.lib.mrcm_profile(self.handle, int(bool(enable))), self.handle)

    def profile_report(self):
        """{kernel: (launches, total_ms)} since profile() and the launch count; clears both."""
        buf = C.create_string_buffer(1 << 16)
        n = C.c_longlong()
        L.check(self.lib.mrcm_profile_report(self.handle, buf, C.c_size_t(len(buf)), C.byref(n)), self.handle)
        out = {}
        for line in buf.value.decode().splitlines():
            name, cnt, ms = line.split()
            out[name] = (int(cnt), float(ms))
        return out, int(n.value)

    # ------------------------------------------------------------------ inspection
    def read_status(self):
        v = [C.c_int() for _ in range(4)]
        code = self.lib.mrcm_read_status(self.handle, self.ws_ptr, *[C.byref(x) for x in v])
        return code, {"not_spd": v[0].value, "unconverged": v[1].value, "interface_zero_pivots": v[2].value,
                      "sweeps": v[3].value}

    def read_fallback(self):
        """(subdomains re-solved in FP64 by the fallback, subdomains that needed it and could not have it)."""
        a, b = C.c_int(), C.c_int()
        L.check(self.lib.mrcm_read_fallback(self.handle, self.ws_ptr, C.byref(a), C.byref(b)), self.handle)
        return int(a.value), int(b.value)

    def read_work(self):
        """MBF entries swept by the refinement sweeps of the last solve."""
        v = C.c_longlong()
        L.check(self.lib.mrcm_read_work(self.handle, self.ws_ptr, C.byref(v)), self.handle)
        return int(v.value)

    def local_ldl_flops(self):
        """(factor flops, all-columns solve flops) of the paper's sparse local LDL^T (minimum degree)."""
        a, b = C.c_double(), C.c_double()
        L.check(self.lib.mrcm_query_local_ldl(self.handle, C.byref(a), C.byref(b)), self.handle)
        return float(a.value), float(b.value)

    def basis(self, i):
        v = [C.c_int() for _ in range(4)]
        L.check(self.lib.mrcm_query_basis(self.handle, int(i), *[C.byref(x) for x in v]), self.handle)
        return tuple(x.value for x in v)

    def export(self, what, sub=0, count=None, dtype="float64"):
        import numpy as np
        if count is None:
            raise ValueError("count required")
        out = np.empty(count, dtype=dtype)
        L.check(self.lib.mrcm_export(self.handle, self.ws_ptr, int(what), int(sub),
                                     out.ctypes.data_as(C.c_void_p), C.c_size_t(out.nbytes)), self.handle)
        return out

    def interface_csr(self):
        """(rowptr, colidx, values, b) of A^int after mrcm_assemble_interface."""
        nd = self.n_interface
        nnz = int(self.sizes["nnz_interface"])
        rowptr = self.export(2, count=nd + 1, dtype="int32")
        colidx = self.export(3, count=nnz, dtype="int32")
        val = self.export(0, count=nnz)
        b = self.export(1, count=nd)
        return rowptr, colidx, val, b

    def mbf_block(self, sub, m, n_cells):
        """MBF columns of one subdomain, (m, n_cells) with cells in box-lexicographic order."""
        return self.export(4, sub=sub, count=m * n_cells).reshape(m, n_cells)
