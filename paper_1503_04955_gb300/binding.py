"""Thin ctypes binding of libdkss.so (include/dkss.h), argument marshalling only.

Every step of a product runs in the library's CUDA kernels; this module only
converts tensors to pointers and status codes to exceptions.  PyTorch supplies
device memory and streams.  A missing or unloadable library raises at import
of the first call: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import buildlib as _build

_lib = None

DKSS_OK = 0
STATUS_NAMES = ["DKSS_OK", "DKSS_EINVAL", "DKSS_EPARAM", "DKSS_ENOMEM", "DKSS_EUNSUPPORTED",
                "DKSS_ECUDA", "DKSS_ETIMEOUT", "DKSS_EDEVICE"]
FORM_IMAD = 1
FORM_INT8TC = 2

# Names exported by libdkss.so (include/dkss.h)
EXPORTS = ["dkss_plan", "dkss_mul", "dkss_sqr", "dkss_ll_step", "dkss_mul_host", "dkss_forward", "dkss_mul_batch",
           "dkss_plan_info", "dkss_plan_rho", "dkss_profile_read", "dkss_plan_launches", "dkss_sync_status", "dkss_plan_destroy",
           "dkss_status_str", "dkss_decode_static", "dkss_batch_plan", "dkss_batch_run", "dkss_batch_job_params",
           "dkss_batch_destroy", "dkss_plan_candidates", "dkss_mlp_forward", "dkss_mlp_grad", "dkss_mlp_adam",
           "dkss_fault_inject", "dkss_plan_choose", "dkss_plan_proth", "dkss_plan_proth_rho", "dkss_proth_ring"]
FORM_PROFILE = 4
RMUL_DIRECT = 16
LEVELS_EVAL = 128
ARITH_MONT = 512       # m = 64 over p^4: 26-bit-limb Montgomery products instead of p-adic digits
DEBUG_CHECKS = 8
TUNE_RULE = 32         # dkss_plan with M..z = 0: the thesis's rule without timing
FAULT_RHO, FAULT_HOST_ALLOC, FAULT_RANGE = 1, 2, 4
PROFILE_KINDS = ["fwd_dft", "fwd_twiddle", "final_pointwise", "inv_twiddle", "inv_dft", "decode"]


class DkssError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        name = STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else str(code)
        super().__init__("%s: %s (%s)" % (what, name, load().dkss_status_str(code).decode()))


def lib_path():
    return _build.lib_path()


def load():
    """Load libdkss.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError("libdkss.so is not built (%s); run __graft_entry__.build() "
                           "or python paper_1503_04955_gb300/buildlib.py" % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    u64, u32, sz = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_size_t
    lib.dkss_plan.argtypes = [ctypes.POINTER(P), u64, u64, u32, u32, u64, u32, u32]
    lib.dkss_mul.argtypes = [P, P, P, P, P]
    lib.dkss_mul_host.argtypes = [P, P, P, P, P]
    lib.dkss_sqr.argtypes = [P, P, P, P]
    lib.dkss_ll_step.argtypes = [P, P, u32, P]
    lib.dkss_forward.argtypes = [P, P, P, P]
    lib.dkss_mul_batch.argtypes = [P, sz, u32, P]
    lib.dkss_plan_info.argtypes = [P, P, sz, P]
    lib.dkss_plan_rho.argtypes = [u64, u64, u32, u32, u64, u32, P, P, sz]
    lib.dkss_profile_read.argtypes = [P, P, P, sz]
    lib.dkss_decode_static.argtypes = [P, u64, u64, u32, u32, u32, P, P]
    lib.dkss_plan_candidates.argtypes = [u64, P, sz, P]
    lib.dkss_plan_candidates.restype = ctypes.c_int
    lib.dkss_plan_choose.argtypes = [u64, u32, P]
    lib.dkss_plan_choose.restype = ctypes.c_int
    lib.dkss_plan_proth.argtypes = [ctypes.POINTER(P), u64, u64, u32, u32, u64, u32, u32]
    lib.dkss_plan_proth_rho.argtypes = [u64, u64, u32, u32, u64, u32, P, P, sz]
    lib.dkss_proth_ring.argtypes = [u64, u64, u32, u32, ctypes.POINTER(u64), ctypes.POINTER(u32)]
    for f in (lib.dkss_plan_proth, lib.dkss_plan_proth_rho, lib.dkss_proth_ring):
        f.restype = ctypes.c_int
    lib.dkss_mlp_forward.argtypes = [P, P, sz, P, P]
    lib.dkss_mlp_grad.argtypes = [P, P, P, sz, P, P, P]
    lib.dkss_mlp_adam.argtypes = [P, P, P, P, ctypes.c_float, u32, P]
    for f in (lib.dkss_mlp_forward, lib.dkss_mlp_grad, lib.dkss_mlp_adam):
        f.restype = ctypes.c_int
    lib.dkss_decode_static.restype = ctypes.c_int
    lib.dkss_fault_inject.argtypes = [u32]
    lib.dkss_fault_inject.restype = u32
    lib.dkss_plan_launches.argtypes = [P]
    lib.dkss_plan_launches.restype = u32
    lib.dkss_sync_status.argtypes = [P, P]
    lib.dkss_plan_destroy.argtypes = [P]
    lib.dkss_status_str.argtypes = [ctypes.c_int]
    lib.dkss_status_str.restype = ctypes.c_char_p
    for name in ("dkss_plan", "dkss_mul", "dkss_sqr", "dkss_ll_step", "dkss_mul_host", "dkss_forward", "dkss_mul_batch",
                 "dkss_plan_info", "dkss_plan_rho", "dkss_profile_read", "dkss_sync_status", "dkss_plan_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code, what):
    if code != DKSS_OK:
        raise DkssError(code, what)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _words2_to_ints(arr):
    arr = np.asarray(arr, dtype=np.uint64)
    return [int(lo) | (int(hi) << 64) for lo, hi in zip(arr[0::2], arr[1::2])]


N_CONSTS = 25
CONST_NAMES = ["P2", "mu", "L", "levels", "pz_lo", "pz_hi", "zeta", "omega_lo", "omega_hi", "gamma_lo", "gamma_hi",
               "LR", "rmul", "prescale", "eval_ok", "eval_skip", "M", "m", "u", "p_lo", "z", "p_hi", "sparse", "dev_bytes",
               "padic"]
RMUL_FORMS = ("ntt", "direct", "int8tc", "eval")     # consts["rmul"] indexes this


def _consts_dict(c):
    d = dict(zip(CONST_NAMES, [int(x) for x in c]))
    d["pz"] = d.pop("pz_lo") | (d.pop("pz_hi") << 64)
    d["omega"] = d.pop("omega_lo") | (d.pop("omega_hi") << 64)
    d["gamma"] = d.pop("gamma_lo") | (d.pop("gamma_hi") << 64)
    d["p"] = d.pop("p_lo") | (d.pop("p_hi") << 64)
    return d


def plan_choose(n_bits, flags=TUNE_RULE):
    """(M, m, u, p, z) that dkss_plan chooses for N-bit operands (dkss_plan_choose);
    with TUNE_RULE the thesis's rule on the host alone."""
    out = np.zeros(5, dtype=np.uint64)
    _check(load().dkss_plan_choose(n_bits, flags, out.ctypes.data), "dkss_plan_choose")
    return tuple(int(x) for x in out)


def proth_ring(n_bits, M, m, u):
    """(h, n) of the Proth ring with the cheap reduction for these parameters (dkss_proth_ring)."""
    h, n = ctypes.c_uint64(), ctypes.c_uint32()
    _check(load().dkss_proth_ring(n_bits, M, m, u, ctypes.byref(h), ctypes.byref(n)), "dkss_proth_ring")
    return int(h.value), int(n.value)


def plan_proth_rho(n_bits, M, m, u, h, n):
    lib = load()
    rho = np.zeros(2 * m, dtype=np.uint64)
    consts = np.zeros(N_CONSTS, dtype=np.uint64)
    _check(lib.dkss_plan_proth_rho(n_bits, M, m, u, h, n, rho.ctypes.data, consts.ctypes.data, N_CONSTS),
           "dkss_plan_proth_rho")
    return _words2_to_ints(rho), _consts_dict(consts)


def plan_rho(n_bits, M, m, u, p, z):
    """Host-only plan math: (rho coefficients, constants dict)."""
    lib = load()
    rho = np.zeros(2 * m, dtype=np.uint64)
    consts = np.zeros(N_CONSTS, dtype=np.uint64)
    _check(lib.dkss_plan_rho(n_bits, M, m, u, p, z, rho.ctypes.data, consts.ctypes.data, N_CONSTS), "dkss_plan_rho")
    return _words2_to_ints(rho), _consts_dict(consts)


class Plan:
    """A DKSS_MUL plan for N-bit operands (dkss_plan).  With M = m = u = p = z = 0
    (the defaults) the library chooses the parameters (rule and measurement)."""

    def __init__(self, n_bits, M=0, m=0, u=0, p=0, z=0, flags=0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.dkss_plan(ctypes.byref(h), n_bits, M, m, u, p, z, flags), "dkss_plan")
        self._h = h
        self.n_bits = n_bits
        if M == m == u == p == z == 0:
            consts = np.zeros(N_CONSTS, dtype=np.uint64)
            _check(lib.dkss_plan_info(h, consts.ctypes.data, N_CONSTS, None), "dkss_plan_info")
            M, m, u, p, z = (int(x) for x in consts[16:21])
        self.M, self.m, self.u, self.p, self.z = M, m, u, p, z
        self.words = (n_bits + 63) // 64

    @classmethod
    def proth(cls, n_bits, M, m, u, h, n, flags=0):
        """Plan over Z/pZ with the Proth prime p = h 2^n + 1 (dkss_plan_proth)."""
        lib = load()
        hd = ctypes.c_void_p()
        _check(lib.dkss_plan_proth(ctypes.byref(hd), n_bits, M, m, u, h, n, flags), "dkss_plan_proth")
        self = cls.__new__(cls)
        self._h = hd
        self.n_bits, self.M, self.m, self.u, self.p, self.z = n_bits, M, m, u, (h << n) + 1, 1
        self.words = (n_bits + 63) // 64
        return self

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().dkss_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self):
        consts = np.zeros(N_CONSTS, dtype=np.uint64)
        rho = np.zeros(2 * self.m, dtype=np.uint64)
        _check(load().dkss_plan_info(self._h, consts.ctypes.data, N_CONSTS, rho.ctypes.data), "dkss_plan_info")
        d = _consts_dict(consts)
        d["rho"] = _words2_to_ints(rho)
        return d

    @property
    def launches(self):
        return int(load().dkss_plan_launches(self._h))

    def _check_operand(self, t, n):
        if not t.is_cuda or t.element_size() != 8 or not t.is_contiguous() or t.numel() != n:
            raise ValueError("expected a contiguous CUDA tensor of %d 64-bit words" % n)

    def mul(self, a, b, out=None, stream=None):
        """out = a*b on the GPU; a, b, out: CUDA tensors of 64-bit words (int64/uint64)."""
        import torch
        self._check_operand(a, self.words)
        self._check_operand(b, self.words)
        if out is None:
            out = torch.empty(2 * self.words, dtype=a.dtype, device=a.device)
        self._check_operand(out, 2 * self.words)
        _check(load().dkss_mul(self._h, a.data_ptr(), b.data_ptr(), out.data_ptr(), _stream_handle(stream)),
               "dkss_mul")
        return out

    def sqr(self, a, out=None, stream=None):
        """out = a*a on the GPU (dkss_sqr: one forward transform)."""
        import torch
        self._check_operand(a, self.words)
        if out is None:
            out = torch.empty(2 * self.words, dtype=a.dtype, device=a.device)
        self._check_operand(out, 2 * self.words)
        _check(load().dkss_sqr(self._h, a.data_ptr(), out.data_ptr(), _stream_handle(stream)), "dkss_sqr")
        return out

    def mul_host(self, a, b, out=None, stream=None):
        """Product of host arrays (numpy uint64) through dkss_mul_host."""
        a = np.ascontiguousarray(a, dtype=np.uint64)
        b = np.ascontiguousarray(b, dtype=np.uint64)
        if a.size != self.words or b.size != self.words:
            raise ValueError("operands must have %d words" % self.words)
        if out is None:
            out = np.empty(2 * self.words, dtype=np.uint64)
        _check(load().dkss_mul_host(self._h, a.ctypes.data, b.ctypes.data, out.ctypes.data,
                                    _stream_handle(stream)), "dkss_mul_host")
        return out

    def forward(self, a, stream=None):
        """Forward transform a(rho^i), natural order: tensor (2M, m, 2) of 64-bit words."""
        import torch
        self._check_operand(a, self.words)
        out = torch.empty((2 * self.M, self.m, 2), dtype=torch.int64, device=a.device)
        _check(load().dkss_forward(self._h, a.data_ptr(), out.data_ptr(), _stream_handle(stream)), "dkss_forward")
        return out

    def profile_read(self):
        """{kind: (total ms, groups timed)} since the last read (plan built with FORM_PROFILE)."""
        ms = np.zeros(8, dtype=np.float64)
        cnt = np.zeros(8, dtype=np.uint64)
        _check(load().dkss_profile_read(self._h, ms.ctypes.data, cnt.ctypes.data, 8), "dkss_profile_read")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROFILE_KINDS)}

    def sync_status(self, stream=None):
        _check(load().dkss_sync_status(self._h, _stream_handle(stream)), "device status")


def decode_static(c, n_bits, M, m, u, L, out=None, stream=None):
    """dkss_decode_static: product words from a product polynomial without any
    allocation inside the library.  c: CUDA tensor of 2M*m*L 32-bit words
    (int32/uint32); out: CUDA tensor of 2*ceil(N/64) 64-bit words."""
    import torch
    words = (n_bits + 63) // 64
    if out is None:
        out = torch.empty(2 * words, dtype=torch.int64, device=c.device)
    if not c.is_cuda or c.element_size() != 4 or not c.is_contiguous() or c.numel() != 2 * M * m * L:
        raise ValueError("c must be a contiguous CUDA tensor of 2M*m*L 32-bit words")
    if not out.is_cuda or out.element_size() != 8 or not out.is_contiguous() or out.numel() != 2 * words:
        raise ValueError("out must be a contiguous CUDA tensor of 2*ceil(N/64) 64-bit words")
    _check(load().dkss_decode_static(c.data_ptr(), n_bits, M, m, u, L, out.data_ptr(), _stream_handle(stream)),
           "dkss_decode_static")
    return out


def ll_step(c, s, p, stream=None):
    """dkss_ll_step: s = (c - 2) mod (2^p - 1), the Lucas-Lehmer step after the
    square.  c: CUDA tensor of 2*ceil(p/64) 64-bit words; s: ceil(p/64) words."""
    w = (p + 63) // 64
    for t, n in ((c, 2 * w), (s, w)):
        if not t.is_cuda or t.element_size() != 8 or not t.is_contiguous() or t.numel() != n:
            raise ValueError("expected a contiguous CUDA tensor of %d 64-bit words" % n)
    _check(load().dkss_ll_step(c.data_ptr(), s.data_ptr(), p, _stream_handle(stream)), "dkss_ll_step")
    return s


BATCH_RULE = 32
BATCH_NO_GRAPH = 64
BATCH_PROTH = 128
BATCH_NO_PROTH = 256


class _Job(ctypes.Structure):
    _fields_ = [("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n_bits", ctypes.c_uint64)]


def _load_batch():
    lib = load()
    if not getattr(lib, "_batch_ready", False):
        P = ctypes.c_void_p
        lib.dkss_batch_plan.argtypes = [ctypes.POINTER(P), P, ctypes.c_size_t, ctypes.c_uint32]
        lib.dkss_batch_run.argtypes = [P, P, P]
        lib.dkss_batch_job_params.argtypes = [P, ctypes.c_size_t, P, ctypes.c_size_t]
        lib.dkss_batch_destroy.argtypes = [P]
        lib.dkss_mul_batch.argtypes = [P, ctypes.c_size_t, ctypes.c_uint32, P]
        for f in (lib.dkss_batch_plan, lib.dkss_batch_run, lib.dkss_batch_job_params, lib.dkss_batch_destroy,
                  lib.dkss_mul_batch):
            f.restype = ctypes.c_int
        lib._batch_ready = True
    return lib


def _jobs_array(a_list, b_list, out_list, n_bits):
    jobs = (_Job * len(n_bits))()
    for j, (a, b, o, n) in enumerate(zip(a_list, b_list, out_list, n_bits)):
        jobs[j].a, jobs[j].b, jobs[j].out, jobs[j].n_bits = a.data_ptr(), b.data_ptr(), o.data_ptr(), int(n)
    return jobs


class Batch:
    """A planned batch of products of uneven sizes (dkss_batch_plan)."""

    PARAM_NAMES = ["M", "m", "u", "p_lo", "z", "class_bits", "levels", "grid", "graph", "p_hi", "proth", "h", "n"]

    def __init__(self, n_bits, flags=0):
        lib = _load_batch()
        self.n_bits = [int(n) for n in n_bits]
        arr = (ctypes.c_uint64 * len(self.n_bits))(*self.n_bits)
        h = ctypes.c_void_p()
        _check(lib.dkss_batch_plan(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), len(self.n_bits), flags),
               "dkss_batch_plan")
        self._h = h

    def job_params(self, j):
        v = np.zeros(13, dtype=np.uint64)
        _check(_load_batch().dkss_batch_job_params(self._h, j, v.ctypes.data, 13), "dkss_batch_job_params")
        d = dict(zip(self.PARAM_NAMES, [int(x) for x in v]))
        d["p"] = d.pop("p_lo") | (d.pop("p_hi") << 64)
        return d

    def class_plan(self, j, n_bits=None):
        """A single-product plan with job j's class parameters (for comparison)."""
        d = self.job_params(j)
        n_bits = n_bits or self.n_bits[j]
        if d["proth"]:
            return Plan.proth(n_bits, d["M"], d["m"], d["u"], d["h"], d["n"])
        return Plan(n_bits, d["M"], d["m"], d["u"], d["p"], d["z"])

    def run(self, a_list, b_list, out_list, stream=None):
        """out_list[j] = a_list[j] * b_list[j] (CUDA tensors of 64-bit words)."""
        jobs = _jobs_array(a_list, b_list, out_list, self.n_bits)
        self._jobs = jobs   # keep alive until the host-to-device copy is done
        _check(_load_batch().dkss_batch_run(self._h, ctypes.cast(jobs, ctypes.c_void_p), _stream_handle(stream)),
               "dkss_batch_run")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _load_batch().dkss_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def mul_batch(a_list, b_list, out_list, n_bits, flags=0, stream=None):
    """dkss_mul_batch: plan (cached while the lengths repeat) and run in one call."""
    jobs = _jobs_array(a_list, b_list, out_list, n_bits)
    _check(_load_batch().dkss_mul_batch(ctypes.cast(jobs, ctypes.c_void_p), len(n_bits), flags,
                                        _stream_handle(stream)), "dkss_mul_batch")


CANDIDATE_FIELDS = ["M", "m", "u", "p", "z", "L", "LR", "levels", "r_last", "P2"]


def plan_candidates(n_bits):
    """dkss_plan_candidates: list of dicts of valid parameter sets for N-bit operands."""
    lib = load()
    n = ctypes.c_size_t()
    _check(lib.dkss_plan_candidates(n_bits, None, 0, ctypes.byref(n)), "dkss_plan_candidates")
    rows = np.zeros(10 * max(1, n.value), dtype=np.uint64)
    _check(lib.dkss_plan_candidates(n_bits, rows.ctypes.data, n.value, ctypes.byref(n)), "dkss_plan_candidates")
    return [dict(zip(CANDIDATE_FIELDS, [int(v) for v in rows[10 * i:10 * i + 10]])) for i in range(n.value)]
