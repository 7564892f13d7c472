"""GB300 sparse-FCI sigma = H psi: a thin ctypes binding over libsfci.so.

Every function here marshals arguments to the C ABI declared in
``include/sfci.h`` and returns torch tensors on the current CUDA device; all
arithmetic runs in the library's CUDA kernels.  There is no CPU path: if the
library is not built, or no GPU is present, the calls raise.

Vectors are (rank, coef) pairs: ranks are stored in int64 tensors holding the
bit pattern of the library's uint64 ranks, coefficients in float64.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsfci.so")

SFCI_OK, SFCI_E_INVALID, SFCI_E_CAPACITY, SFCI_E_OVERFLOW = 0, 1, 2, 3
SFCI_E_CUDA, SFCI_E_TIMEOUT, SFCI_E_NOMEM = 4, 5, 6
SFCI_FP32_ELEMENTS = 1  # sfci_system_create flag: float32 off-diagonal elements
SFCI_LZ_FALLBACK_STRESS = 1  # sfci_params flag (tests): 2048-element buckets in 1024-slot tables


class SfciError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"sfci status {status}: {message}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("n_keep", C.c_int64), ("table_capacity", C.c_int64),
                ("eps_screen", C.c_double), ("conv_tol", C.c_double),
                ("n_lanczos", C.c_int32), ("max_iter", C.c_int32),
                ("flags", C.c_uint32), ("bucket_elems", C.c_int32),
                ("mem_budget", C.c_int64), ("emit_warps", C.c_int32), ("ovf_max_log2", C.c_int32),
                ("eps_element", C.c_double)]


class StepInfo(C.Structure):
    _fields_ = [("iter", C.c_int32), ("cycle", C.c_int32), ("index", C.c_int32),
                ("cycle_end", C.c_int32), ("converged", C.c_int32), ("breakdown", C.c_int32),
                ("lambda_min", C.c_double), ("a", C.c_double), ("b", C.c_double),
                ("u_norm", C.c_double), ("t00", C.c_double),
                ("n_in", C.c_int64), ("n_sigma", C.c_int64), ("n_kept", C.c_int64),
                ("n_elements", C.c_int64), ("n_psi", C.c_int64),
                ("ms_sigma", C.c_double), ("ms_step", C.c_double),
                ("ms_emit", C.c_double), ("ms_merge", C.c_double),
                ("ms_plan", C.c_double), ("ms_topk", C.c_double),
                ("n_passes", C.c_int32), ("n_buckets_log2", C.c_int32),
                ("tau", C.c_double), ("cut", C.c_double), ("redo", C.c_int32), ("bucket_redo", C.c_int32),
                ("pass_budget_gb", C.c_double), ("regions_gb", C.c_double), ("free_gb", C.c_double),
                ("n_overflow", C.c_int64), ("ms_alloc", C.c_double), ("n_emitted", C.c_int64),
                ("n_alpha_runs", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
_vp, _i64, _u64, _f64, _i32 = C.c_void_p, C.c_int64, C.c_uint64, C.c_double, C.c_int


def lib():
    """Load libsfci.so; raise if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2312_01846_gb300.build` (needs nvcc)")
    L = C.CDLL(LIB_PATH)
    sig = {
        "sfci_status_string": (C.c_char_p, [_i32]),
        "sfci_last_error": (C.c_char_p, []),
        "sfci_version": (_i32, []),
        "sfci_kernel_launches": (_i64, []),
        "sfci_lanczos_load": (_i32, [_vp, _vp, _vp, _i64]),
        "sfci_lanczos_set_input": (_i32, [_vp, _vp, _vp, _i64]),
        "sfci_system_create": (_i32, [C.POINTER(_vp), _i32, _i32, _i32, _vp, _vp, _f64, C.c_uint32]),
        "sfci_system_destroy": (_i32, [_vp]),
        "sfci_dim": (_i32, [_vp, C.POINTER(_u64)]),
        "sfci_n_connected": (_i32, [_vp, C.POINTER(_i64)]),
        "sfci_rank": (_i32, [_vp, _vp, _vp, _vp, _i64, _vp]),
        "sfci_unrank": (_i32, [_vp, _vp, _vp, _vp, _i64, _vp]),
        "sfci_sigma_workspace_bytes": (_i32, [_vp, _i64, _i64, C.POINTER(C.c_size_t)]),
        "sfci_sigma": (_i32, [_vp, _vp, _vp, _i64, _f64, _vp, _vp, _i64, C.POINTER(_i64), _vp,
                              C.c_size_t, _vp]),
        "sfci_truncate_topk_workspace_bytes": (_i32, [_i64, _i64, C.POINTER(C.c_size_t)]),
        "sfci_truncate_topk": (_i32, [_vp, _vp, _i64, _i64, _i32, _vp, _vp, C.POINTER(_i64), _vp,
                                      C.c_size_t, _vp]),
        "sfci_truncate_topk_noalloc": (_i32, [_vp, _vp, _i64, _i64, _i32, _vp, _vp, C.POINTER(_i64),
                                              _vp]),
        "sfci_lanczos_create": (_i32, [C.POINTER(_vp), _vp, C.POINTER(Params), _vp, _vp, _i64, _vp]),
        "sfci_lanczos_step": (_i32, [_vp, C.POINTER(StepInfo)]),
        "sfci_lanczos_vector": (_i32, [_vp, _vp, _vp, _i64, C.POINTER(_i64)]),
        "sfci_lanczos_matrices": (_i32, [_vp, _vp, _vp]),
        "sfci_lanczos_destroy": (_i32, [_vp]),
        "sfci_rdm12_workspace_bytes": (_i32, [_vp, _i64, C.POINTER(C.c_size_t)]),
        "sfci_rdm12": (_i32, [_vp, _vp, _vp, _i64, _vp, _vp, C.POINTER(_f64), _vp, C.c_size_t, _vp]),
        "sfci_rdm_energy": (_i32, [_i32, _vp, _vp, _f64, _vp, _vp, _f64, C.POINTER(_f64), _vp, C.c_size_t,
                                   _vp]),
        "sfci_debug_pipe_rate": (_i32, [_i32, _i64, _vp, C.POINTER(_f64), _vp]),
        "sfci_debug_excitations": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _i64, C.POINTER(_i64), _vp]),
        "sfci_scan_create": (_i32, [C.POINTER(_vp), _i32, C.POINTER(_vp), C.POINTER(Params),
                                    C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_i64), _i32]),
        "sfci_scan_step": (_i32, [_vp, C.POINTER(StepInfo)]),
        "sfci_scan_solver": (_i32, [_vp, _i32, C.POINTER(_vp)]),
        "sfci_scan_destroy": (_i32, [_vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _LIB = L
    return L


def _check(st, what):
    if st != SFCI_OK:
        msg = lib().sfci_last_error().decode()
        raise SfciError(st, f"{what}: {msg}")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _dev(x, dtype):
    """Contiguous tensor of `dtype` on the current CUDA device (uint64 numpy
    arrays are taken bit for bit)."""
    if not torch.is_tensor(x):
        import numpy as np
        a = np.ascontiguousarray(x)
        if a.dtype == np.uint64:
            a = a.view(np.int64)
        x = torch.from_numpy(a)
    return x.to(device="cuda", dtype=dtype).contiguous()


class System:
    """Integrals + electron counts on the device (sfci_system_create)."""

    def __init__(self, n, na, nb, h, g, e_core=0.0, flags=0):
        """flags: 0 or SFCI_FP32_ELEMENTS (float32 off-diagonal elements)."""
        import numpy as np
        self.n, self.na, self.nb = int(n), int(na), int(nb)
        self.flags = int(flags)
        self._h = np.ascontiguousarray(np.asarray(h, dtype=np.float64).reshape(n, n))
        self._g = np.ascontiguousarray(np.asarray(g, dtype=np.float64).reshape(n, n, n, n))
        self.e_core = float(e_core)
        h_ = C.c_void_p()
        torch.cuda.init()
        _check(lib().sfci_system_create(C.byref(h_), self.n, self.na, self.nb,
                                        self._h.ctypes.data, self._g.ctypes.data,
                                        self.e_core, self.flags), "sfci_system_create")
        self.handle = h_
        d = C.c_uint64()
        _check(lib().sfci_dim(self.handle, C.byref(d)), "sfci_dim")
        self.dim = int(d.value)
        nc = C.c_int64()
        _check(lib().sfci_n_connected(self.handle, C.byref(nc)), "sfci_n_connected")
        self.n_conn = int(nc.value)

    @classmethod
    def from_dict(cls, d, flags=0):
        return cls(d["n"], d["na"], d["nb"], d["h"], d["g"], d.get("e_core", 0.0), flags)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().sfci_system_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfci_rank(sys: System, alpha, beta, stream=None):
    a = _dev(alpha, torch.int64)
    b = _dev(beta, torch.int64)
    r = torch.empty_like(a)
    _check(lib().sfci_rank(sys.handle, _ptr(a), _ptr(b), _ptr(r), a.numel(), _stream(stream)),
           "sfci_rank")
    return r


def sfci_unrank(sys: System, rank, stream=None):
    r = _dev(rank, torch.int64)
    a = torch.empty_like(r)
    b = torch.empty_like(r)
    _check(lib().sfci_unrank(sys.handle, _ptr(r), _ptr(a), _ptr(b), r.numel(), _stream(stream)),
           "sfci_unrank")
    return a, b


def sigma_workspace_bytes(sys: System, n_in, out_cap):
    nb = C.c_size_t()
    _check(lib().sfci_sigma_workspace_bytes(sys.handle, int(n_in), int(out_cap), C.byref(nb)),
           "sfci_sigma_workspace_bytes")
    return int(nb.value)


def sfci_sigma(sys: System, rank, coef, eps_screen=0.0, out_cap=None, stream=None):
    """sigma = H psi; returns (rank, coef) ascending by rank.  If out_cap is not
    given it starts from min(n_in * (n_conn + 1), 2^24) and grows on
    SFCI_E_CAPACITY."""
    r = _dev(rank, torch.int64)
    c = _dev(coef, torch.float64)
    if out_cap is not None:
        cap = int(out_cap)
    else:
        cap = max(1024, min(r.numel() * (sys.n_conn + 1), 1 << 24))
    for _ in range(16):
        ws = torch.empty(sigma_workspace_bytes(sys, r.numel(), cap), dtype=torch.uint8, device="cuda")
        orank = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
        ocoef = torch.empty(max(cap, 1), dtype=torch.float64, device="cuda")
        n = C.c_int64()
        st = lib().sfci_sigma(sys.handle, _ptr(r), _ptr(c), r.numel(), float(eps_screen),
                              _ptr(orank), _ptr(ocoef), cap, C.byref(n), _ptr(ws), ws.numel(),
                              _stream(stream))
        if st == SFCI_E_CAPACITY and n.value > cap:
            del ws, orank, ocoef
            cap = max(int(n.value * 1.25) + 1024, 4 * cap)
            continue
        _check(st, "sfci_sigma")
        return orank[: n.value], ocoef[: n.value]
    raise SfciError(SFCI_E_CAPACITY, "sfci_sigma: output keeps growing")


def sfci_truncate_topk(rank, coef, k, normalize=True, stream=None):
    r = _dev(rank, torch.int64)
    c = _dev(coef, torch.float64)
    k = int(k)
    nb = C.c_size_t()
    _check(lib().sfci_truncate_topk_workspace_bytes(r.numel(), k, C.byref(nb)),
           "sfci_truncate_topk_workspace_bytes")
    ws = torch.empty(int(nb.value), dtype=torch.uint8, device="cuda")
    orank = torch.empty(max(k, 1), dtype=torch.int64, device="cuda")
    ocoef = torch.empty(max(k, 1), dtype=torch.float64, device="cuda")
    n = C.c_int64()
    _check(lib().sfci_truncate_topk(_ptr(r), _ptr(c), r.numel(), k, int(bool(normalize)),
                                    _ptr(orank), _ptr(ocoef), C.byref(n), _ptr(ws), ws.numel(),
                                    _stream(stream)), "sfci_truncate_topk")
    return orank[: n.value], ocoef[: n.value]


def sfci_truncate_topk_noalloc(rank, coef, k, normalize=True, out_rank=None, out_coef=None,
                               stream=None):
    """sfci_truncate_topk through the entry point that allocates nothing on the
    device (fixed 20 MiB scratch inside the library, k <= 2^20).  Pass
    out_rank/out_coef (device, >= k entries) to keep the call free of
    allocations here too; calls that overlap in time must not share a device."""
    r = _dev(rank, torch.int64)
    c = _dev(coef, torch.float64)
    k = int(k)
    if out_rank is None:
        out_rank = torch.empty(max(k, 1), dtype=torch.int64, device="cuda")
    if out_coef is None:
        out_coef = torch.empty(max(k, 1), dtype=torch.float64, device="cuda")
    if out_rank.numel() < k or out_coef.numel() < k:
        raise ValueError("output buffers need room for k entries")
    n = C.c_int64()
    _check(lib().sfci_truncate_topk_noalloc(_ptr(r), _ptr(c), r.numel(), k, int(bool(normalize)),
                                            _ptr(out_rank), _ptr(out_coef), C.byref(n),
                                            _stream(stream)), "sfci_truncate_topk_noalloc")
    return out_rank[: n.value], out_coef[: n.value]


def sfci_debug_excitations(sys: System, rank, stream=None):
    r = _dev(rank, torch.int64)
    m = r.numel() * (sys.n_conn + 1)
    src = torch.empty(max(m, 1), dtype=torch.int64, device="cuda")
    tgt = torch.empty(max(m, 1), dtype=torch.int64, device="cuda")
    elem = torch.empty(max(m, 1), dtype=torch.float64, device="cuda")
    n = C.c_int64()
    _check(lib().sfci_debug_excitations(sys.handle, _ptr(r), r.numel(), _ptr(src), _ptr(tgt),
                                        _ptr(elem), m, C.byref(n), _stream(stream)),
           "sfci_debug_excitations")
    return src[:m], tgt[:m], elem[:m]


def sfci_rdm12(sys: System, rank, coef, stream=None):
    """Spin-summed 1- and 2-RDMs of psi (not normalised) and <psi|psi>."""
    r = _dev(rank, torch.int64)
    c = _dev(coef, torch.float64)
    nb = C.c_size_t()
    _check(lib().sfci_rdm12_workspace_bytes(sys.handle, r.numel(), C.byref(nb)),
           "sfci_rdm12_workspace_bytes")
    ws = torch.empty(int(nb.value), dtype=torch.uint8, device="cuda")
    n = sys.n
    g1 = torch.empty((n, n), dtype=torch.float64, device="cuda")
    g2 = torch.empty((n, n, n, n), dtype=torch.float64, device="cuda")
    nrm = C.c_double()
    _check(lib().sfci_rdm12(sys.handle, _ptr(r), _ptr(c), r.numel(), _ptr(g1), _ptr(g2),
                            C.byref(nrm), _ptr(ws), ws.numel(), _stream(stream)), "sfci_rdm12")
    return g1, g2, float(nrm.value)


def sfci_rdm_energy(g1, g2, norm2, h, g, e_core=0.0, stream=None):
    """e_core + (sum h g1 + 1/2 sum g g2) / norm2, contracted in the library."""
    n = g1.shape[0]
    hh = h.detach().to(device="cuda", dtype=torch.float64).contiguous()
    gg = g.detach().to(device="cuda", dtype=torch.float64).contiguous()
    if hh.numel() != n * n or gg.numel() != n ** 4:
        raise ValueError("h must be (n, n) and g (n, n, n, n) for the RDMs' n")
    ws = torch.empty(4096, dtype=torch.uint8, device="cuda")
    e = C.c_double()
    _check(lib().sfci_rdm_energy(n, _ptr(g1), _ptr(g2), float(norm2), _ptr(hh), _ptr(gg), float(e_core),
                                 C.byref(e), _ptr(ws), ws.numel(), _stream(stream)), "sfci_rdm_energy")
    return float(e.value)


class RayleighEnergy(torch.autograd.Function):
    """E(h, g) = e_core + (sum h gamma + 1/2 sum g Gamma) / <psi|psi> for a fixed
    sparse psi; gamma, Gamma come from sfci_rdm12 and E from sfci_rdm_energy,
    so dE/dh = gamma / <psi|psi> and dE/dg = Gamma / (2 <psi|psi>).  h: (n, n),
    g: (n, n, n, n) float64 CUDA tensors; sys fixes n and the electron counts."""

    @staticmethod
    def forward(ctx, h, g, sys, rank, coef, e_core=0.0):
        g1, g2, nrm = sfci_rdm12(sys, rank, coef)
        e = sfci_rdm_energy(g1, g2, nrm, h, g, e_core)
        ctx.nrm = nrm
        ctx.save_for_backward(g1, g2)
        return torch.tensor(e, dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, grad):
        # dE/dh = gamma / <psi|psi>, dE/dg = Gamma / (2 <psi|psi>): a scale of the
        # library's RDMs by the incoming gradient
        g1, g2 = ctx.saved_tensors
        return grad * (g1 / ctx.nrm), grad * (g2 * (0.5 / ctx.nrm)), None, None, None, None


class Lanczos:
    """The SFCI solver (sfci_lanczos_create / _step / _vector / _destroy)."""

    def __init__(self, sys: System, init_rank, init_coef, n_keep, n_lanczos=10, max_iter=0,
                 eps_screen=0.0, conv_tol=0.0, table_capacity=0, bucket_elems=0, stream=None,
                 mem_budget=0, emit_warps=0, eps_element=0.0, ovf_max_log2=0, flags=0):
        self.sys = sys
        r = _dev(init_rank, torch.int64)
        c = _dev(init_coef, torch.float64)
        self.params = Params(int(n_keep), int(table_capacity), float(eps_screen), float(conv_tol),
                             int(n_lanczos), int(max_iter), int(flags), int(bucket_elems),
                             int(mem_budget), int(emit_warps), int(ovf_max_log2), float(eps_element))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib().sfci_lanczos_create(C.byref(h), sys.handle, C.byref(self.params), _ptr(r),
                                         _ptr(c), r.numel(), _stream(self.stream)),
               "sfci_lanczos_create")
        self.handle = h

    def step(self):
        info = StepInfo()
        _check(lib().sfci_lanczos_step(self.handle, C.byref(info)), "sfci_lanczos_step")
        return info.as_dict()

    def load(self, rank, coef):
        """Restart from a new trial vector (sfci_lanczos_load)."""
        r = _dev(rank, torch.int64)
        c = _dev(coef, torch.float64)
        _check(lib().sfci_lanczos_load(self.handle, _ptr(r), _ptr(c), r.numel()),
               "sfci_lanczos_load")

    def set_input(self, rank, coef):
        """Replace the current input vector w_i, keeping the cycle (sfci_lanczos_set_input)."""
        r = _dev(rank, torch.int64)
        c = _dev(coef, torch.float64)
        _check(lib().sfci_lanczos_set_input(self.handle, _ptr(r), _ptr(c), r.numel()),
               "sfci_lanczos_set_input")

    def vector(self):
        cap = int(self.params.n_keep)
        r = torch.empty(cap, dtype=torch.int64, device="cuda")
        c = torch.empty(cap, dtype=torch.float64, device="cuda")
        n = C.c_int64()
        _check(lib().sfci_lanczos_vector(self.handle, _ptr(r), _ptr(c), cap, C.byref(n)),
               "sfci_lanczos_vector")
        return r[: n.value], c[: n.value]

    def matrices(self):
        import numpy as np
        NL = int(self.params.n_lanczos)
        T = np.zeros((NL, NL))
        S = np.zeros((NL, NL))
        _check(lib().sfci_lanczos_matrices(self.handle, T.ctypes.data, S.ctypes.data),
               "sfci_lanczos_matrices")
        return T, S

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().sfci_lanczos_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scan:
    """Many SFCI problems advanced together (sfci_scan_*): one step runs one
    sfci_lanczos_step of every instance, concurrently, each on its own stream.

    instances: list of (System, init_rank, init_coef, n_keep) tuples."""

    def __init__(self, instances, n_lanczos=10, max_iter=0, eps_screen=0.0, bucket_elems=0,
                 emit_warps=0, workers=0, eps_element=0.0):
        k = len(instances)
        self.systems = [inst[0] for inst in instances]
        self._vecs = [(_dev(inst[1], torch.int64), _dev(inst[2], torch.float64)) for inst in instances]
        self.params = (Params * k)(*[
            Params(int(inst[3]), 0, float(eps_screen), 0.0, int(n_lanczos), int(max_iter), 0,
                   int(bucket_elems), 0, int(emit_warps), 0, float(eps_element)) for inst in instances])
        torch.cuda.synchronize()
        sysh = (_vp * k)(*[s.handle.value for s in self.systems])
        rk = (_vp * k)(*[r.data_ptr() for r, _ in self._vecs])
        cf = (_vp * k)(*[c.data_ptr() for _, c in self._vecs])
        nn = (_i64 * k)(*[r.numel() for r, _ in self._vecs])
        h = C.c_void_p()
        _check(lib().sfci_scan_create(C.byref(h), k, sysh, self.params, rk, cf, nn, int(workers)),
               "sfci_scan_create")
        self.handle = h
        self.count = k

    def step(self):
        infos = (StepInfo * self.count)()
        _check(lib().sfci_scan_step(self.handle, infos), "sfci_scan_step")
        return [x.as_dict() for x in infos]

    def vector(self, i):
        z = C.c_void_p()
        _check(lib().sfci_scan_solver(self.handle, int(i), C.byref(z)), "sfci_scan_solver")
        cap = int(self.params[i].n_keep)
        r = torch.empty(cap, dtype=torch.int64, device="cuda")
        c = torch.empty(cap, dtype=torch.float64, device="cuda")
        n = C.c_int64()
        _check(lib().sfci_lanczos_vector(z, _ptr(r), _ptr(c), cap, C.byref(n)), "sfci_lanczos_vector")
        return r[: n.value], c[: n.value]

    def matrices(self, i):
        """T and S of instance i (sfci_lanczos_matrices of its solver)."""
        import numpy as np
        z = C.c_void_p()
        _check(lib().sfci_scan_solver(self.handle, int(i), C.byref(z)), "sfci_scan_solver")
        NL = int(self.params[i].n_lanczos)
        T = np.zeros((NL, NL))
        S = np.zeros((NL, NL))
        _check(lib().sfci_lanczos_matrices(z, T.ctypes.data, S.ctypes.data), "sfci_lanczos_matrices")
        return T, S

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().sfci_scan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PIPE_KINDS = ("fp64_fma", "fp64_add", "fp64_mul", "fp32_fma", "int64_mad", "smem_atomic_add_u64",
              "smem_atomic_add_u32", "smem_cas_u64", "smem_atomic_add_f32")


def pipe_rate(kind, iters=1 << 14, stream=None):
    """Lane operations per second of one pipe operation (sfci_debug_pipe_rate);
    kind: an index or a name of PIPE_KINDS."""
    k = PIPE_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    ws = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = C.c_double()
    _check(lib().sfci_debug_pipe_rate(k, int(iters), _ptr(ws), C.byref(out), _stream(stream)),
           "sfci_debug_pipe_rate")
    return float(out.value)


def kernel_launches():
    """Kernels libsfci.so has launched in this process so far."""
    return int(lib().sfci_kernel_launches())


def to_u64(t):
    """int64 rank tensor -> numpy uint64 array (same bits)."""
    import numpy as np
    return t.detach().cpu().numpy().view(np.uint64)
