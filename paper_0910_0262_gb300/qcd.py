"""Python binding of libqcd (include/qcd.h): argument marshalling only.

Every step of the operator, the solver and the force runs in the CUDA library;
this module passes torch tensors' device pointers and the context's stream
through ctypes.  There is no fallback: if ``libqcd.so`` is missing or no GPU is
present, the calls raise.

``qcd_*`` functions mirror the C ABI one to one; ``CloverWilson`` is a thin
owner of a ``qcd_ctx`` working on torch tensors; ``CloverPseudofermionAction``
is the torch.autograd.Function S(U, phi) = phi^dag (Mhat^dag Mhat)^-1 phi whose
backward is the fermion force.
"""

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library the binding loads: the in-tree build, or the file named by QCD_LIB (for example the
# debug build, libqcd_debug.so)
LIB_PATH = os.environ.get("QCD_LIB") or os.path.join(_HERE, "libqcd.so")

QCD_OK = 0
STATUS = {0: "QCD_OK", 1: "QCD_ERR_ARG", 2: "QCD_ERR_CUDA", 3: "QCD_ERR_NOMEM", 4: "QCD_ERR_STATE",
          5: "QCD_ERR_NOT_POSDEF", 6: "QCD_ERR_NOT_CONVERGED", 7: "QCD_ERR_NAN", 8: "QCD_ERR_TIMEOUT",
          9: "QCD_ERR_COMM"}

QCD_GAUGE_RECON12 = 1
QCD_OP_DSLASH_EO, QCD_OP_DSLASH_OE, QCD_OP_MHAT, QCD_OP_MDAGM, QCD_OP_CLOVER, QCD_OP_CLOVER_INV = range(6)
QCD_FORCE_INPUT_IS_SOLUTION = 1
QCD_FORCE_GRADIENT = 2
QCD_FORCE_CLOVER_DET = 4
QCD_FORCE_ACCUMULATE = 8
QCD_R_STEP_DEFER_CLOVER = 16


class SolverParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("inner_prec", ctypes.c_int),
                ("reliable_every", ctypes.c_int), ("reliable_delta", ctypes.c_double), ("use_x0", ctypes.c_int)]


class SolverStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("true_rel_resid", ctypes.c_double),
                ("b_dot_x", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


# callbacks of a t-slab call (include/qcd.h): the halo exchange and the sum over the ranks
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int)


class SlabComm(ctypes.Structure):
    _fields_ = [("send_lo", ctypes.c_void_p), ("send_hi", ctypes.c_void_p), ("recv_lo", ctypes.c_void_p),
                ("recv_hi", ctypes.c_void_p), ("exchange", EXCHANGE_FN), ("allreduce", ALLREDUCE_FN),
                ("user", ctypes.c_void_p)]


class QCDError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status
        self.message = message


_lib = None
_P = ctypes.c_void_p
_SIGNATURES = {
    "qcd_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int), ctypes.c_double, _P]),
    "qcd_destroy": (ctypes.c_int, [_P]),
    "qcd_load_gauge": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int]),
    "qcd_clover_build": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double]),
    "qcd_dslash": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "qcd_cg_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(SolverParams),
                                    ctypes.POINTER(SolverStats)]),
    "qcd_fermion_force": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(SolverParams),
                                         ctypes.POINTER(SolverStats)]),
    "qcd_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "qcd_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(KernelStat), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "qcd_mhat_static": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "qcd_selftest_barrier_timeout": (ctypes.c_int, [_P]),
    "qcd_selftest_fastdiv": (ctypes.c_longlong, []),
    "qcd_selftest_site_order": (ctypes.c_longlong, []),
    "qcd_clover_logdet": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "qcd_prepare_source": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "qcd_reconstruct_odd": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "qcd_gauge_force": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_int]),
    "qcd_plaquette": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "qcd_kinetic_energy": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_double)]),
    "qcd_update_links": (ctypes.c_int, [_P, _P, _P, ctypes.c_double]),
    "qcd_r_step": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)]),
    "qcd_polyakov": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "qcd_pbp": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(SolverParams), ctypes.POINTER(SolverStats)]),
    "qcd_probe_fma_peak": (ctypes.c_int, [ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]),
    "qcd_probe_copy_bandwidth": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_double)]),
    "qcd_create_slab": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, _P]),
    "qcd_slab_halo_bytes": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "qcd_slab_dslash": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(SlabComm)]),
    "qcd_slab_cg_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(SolverParams),
                                         ctypes.POINTER(SolverStats), ctypes.POINTER(SlabComm)]),
    "qcd_debug_violations": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_int)]),
    "qcd_selftest_debug_index": (ctypes.c_int, [_P]),
    "qcd_local_group_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int]),
    "qcd_local_group_join": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(SlabComm)]),
    "qcd_local_group_abort": (ctypes.c_int, [_P]),
    "qcd_local_group_destroy": (ctypes.c_int, [_P]),
    "qcd_last_error": (ctypes.c_char_p, []),
}


def lib():
    """Load libqcd.so (built in-tree by ``paper_0910_0262_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libqcd.so is not built; run `python -m paper_0910_0262_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != QCD_OK:
        raise QCDError(status, lib().qcd_last_error().decode())
    return status


# ---- one-to-one wrappers of the C ABI ---------------------------------------------------------------------
def qcd_create(dims, t_bc=-1.0, stream=None):
    ctx = _P()
    d = (ctypes.c_int * 4)(*dims)
    _check(lib().qcd_create(ctypes.byref(ctx), d, float(t_bc), stream))
    return ctx


def qcd_destroy(ctx):
    return _check(lib().qcd_destroy(ctx))


def qcd_load_gauge(ctx, U_ptr, on_device, flags=0):
    return _check(lib().qcd_load_gauge(ctx, U_ptr, int(on_device), int(flags)))


def qcd_clover_build(ctx, kappa, csw):
    return _check(lib().qcd_clover_build(ctx, float(kappa), float(csw)))


def qcd_dslash(ctx, out_ptr, in_ptr, op, dagger, precision, nrhs):
    return _check(lib().qcd_dslash(ctx, out_ptr, in_ptr, int(op), int(dagger), int(precision), int(nrhs)))


def qcd_cg_solve(ctx, x_ptr, b_ptr, nrhs, params, stats):
    """Returns the status (QCD_OK or QCD_ERR_NOT_CONVERGED); raises on other errors."""
    s = lib().qcd_cg_solve(ctx, x_ptr, b_ptr, int(nrhs), ctypes.byref(params), stats)
    if s not in (QCD_OK, 6):
        _check(s)
    return s


def qcd_fermion_force(ctx, F_ptr, in_ptr, nrhs, flags, params, stats):
    s = lib().qcd_fermion_force(ctx, F_ptr, in_ptr, int(nrhs), int(flags),
                                ctypes.byref(params) if params is not None else None, stats)
    if s not in (QCD_OK, 6):
        _check(s)
    return s


def qcd_clover_logdet(ctx):
    """(sum over even sites, sum over odd sites) of log det A(x)."""
    out = (ctypes.c_double * 2)()
    _check(lib().qcd_clover_logdet(ctx, out))
    return out[0], out[1]


def qcd_prepare_source(ctx, bhat_ptr, be_ptr, bo_ptr, nrhs):
    return _check(lib().qcd_prepare_source(ctx, bhat_ptr, be_ptr, bo_ptr, int(nrhs)))


def qcd_reconstruct_odd(ctx, xo_ptr, xe_ptr, bo_ptr, nrhs):
    return _check(lib().qcd_reconstruct_odd(ctx, xo_ptr, xe_ptr, bo_ptr, int(nrhs)))


def qcd_gauge_force(ctx, F_ptr, beta, flags=0):
    return _check(lib().qcd_gauge_force(ctx, F_ptr, float(beta), int(flags)))


def qcd_plaquette(ctx):
    out = ctypes.c_double()
    _check(lib().qcd_plaquette(ctx, ctypes.byref(out)))
    return out.value


def qcd_kinetic_energy(ctx, P_ptr):
    out = ctypes.c_double()
    _check(lib().qcd_kinetic_energy(ctx, P_ptr, ctypes.byref(out)))
    return out.value


def qcd_update_links(ctx, U_ptr, P_ptr, eps):
    return _check(lib().qcd_update_links(ctx, U_ptr, P_ptr, float(eps)))


def qcd_r_step(ctx, U_ptr, P_ptr, eta_ptr, nrhs, eps, beta, flags, params, stats):
    s = lib().qcd_r_step(ctx, U_ptr, P_ptr, eta_ptr, int(nrhs), float(eps), float(beta), int(flags),
                         ctypes.byref(params) if params is not None else None, stats)
    if s not in (QCD_OK, 6):
        _check(s)
    return s


def qcd_polyakov(ctx):
    out = (ctypes.c_double * 2)()
    _check(lib().qcd_polyakov(ctx, out))
    return complex(out[0], out[1])


def qcd_pbp(ctx, eta_e_ptr, eta_o_ptr, nrhs, params, stats):
    out = (ctypes.c_double * nrhs)()
    s = lib().qcd_pbp(ctx, eta_e_ptr, eta_o_ptr, int(nrhs), out, ctypes.byref(params), stats)
    if s not in (QCD_OK, 6):
        _check(s)
    return [out[i] for i in range(nrhs)], s


def qcd_profile(ctx, enable):
    return _check(lib().qcd_profile(ctx, int(enable)))


def qcd_profile_read(ctx, max_entries=64):
    arr = (KernelStat * max_entries)()
    n = ctypes.c_int(0)
    _check(lib().qcd_profile_read(ctx, arr, max_entries, ctypes.byref(n)))
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "total_ms": arr[i].total_ms,
             "bytes": arr[i].bytes, "flops": arr[i].flops} for i in range(n.value)]


def qcd_mhat_static(ctx, out_ptr, in_ptr, dagger=0):
    """Mhat (or Mhat^dag) in FP64 on one field with no device allocation (see include/qcd.h)."""
    return _check(lib().qcd_mhat_static(ctx, out_ptr, in_ptr, int(dagger)))


def qcd_selftest_barrier_timeout(ctx):
    """Returns the status of the barrier self-test (QCD_ERR_TIMEOUT = 8 when the wait gave up)."""
    return lib().qcd_selftest_barrier_timeout(ctx)


def qcd_local_group_create(n):
    """An in-process group of n slabs whose exchanges and sums the library makes (see include/qcd.h)."""
    g = _P()
    _check(lib().qcd_local_group_create(ctypes.byref(g), int(n)))
    return g


def qcd_local_group_join(grp, rank, ctx):
    """Rank `rank` of the group is the slab context ctx; returns the SlabComm its calls take."""
    comm = SlabComm()
    _check(lib().qcd_local_group_join(grp, int(rank), ctx, ctypes.byref(comm)))
    return comm


def qcd_local_group_abort(grp):
    _check(lib().qcd_local_group_abort(grp))


def qcd_local_group_destroy(grp):
    _check(lib().qcd_local_group_destroy(grp))


QCD_DBG_SPINOR, QCD_DBG_LINK, QCD_DBG_CLOVER, QCD_DBG_HALO = 1, 2, 4, 8


def qcd_debug_violations(ctx):
    """(violation bits recorded since the last call, 1 for the debug build else 0); clears the bits."""
    v, d = ctypes.c_uint(0), ctypes.c_int(0)
    _check(lib().qcd_debug_violations(ctx, ctypes.byref(v), ctypes.byref(d)))
    return v.value, d.value


def qcd_selftest_debug_index(ctx):
    _check(lib().qcd_selftest_debug_index(ctx))


def qcd_selftest_fastdiv():
    """Mismatches of the kernels' division by a lattice extent against integer division (host only)."""
    return lib().qcd_selftest_fastdiv()


def qcd_selftest_site_order():
    """Lattices on which the staged FP32 kernel's block order is not a permutation (host only)."""
    return lib().qcd_selftest_site_order()


def qcd_probe_fma_peak(precision=64, stream=None):
    """Measured FMA throughput (TFLOP/s) of the current device in FP64 or FP32 (see include/qcd.h)."""
    v = ctypes.c_double()
    _check(lib().qcd_probe_fma_peak(int(precision), stream, ctypes.byref(v)))
    return v.value


def qcd_probe_copy_bandwidth(nbytes, reps=20, stream=None):
    """Measured bandwidth (GB/s, read + write) of a device copy of nbytes (see include/qcd.h)."""
    v = ctypes.c_double()
    _check(lib().qcd_probe_copy_bandwidth(int(nbytes), int(reps), stream, ctypes.byref(v)))
    return v.value


def qcd_create_slab(dims, t_offset, t_local, t_bc=-1.0, stream=None):
    ctx = _P()
    d = (ctypes.c_int * 4)(*dims)
    _check(lib().qcd_create_slab(ctypes.byref(ctx), d, int(t_offset), int(t_local), float(t_bc), stream))
    return ctx


def qcd_slab_halo_bytes(ctx, precision, nrhs):
    n = ctypes.c_size_t()
    _check(lib().qcd_slab_halo_bytes(ctx, int(precision), int(nrhs), ctypes.byref(n)))
    return n.value


def qcd_slab_dslash(ctx, out_ptr, in_ptr, op, dagger, precision, nrhs, comm):
    return _check(lib().qcd_slab_dslash(ctx, out_ptr, in_ptr, int(op), int(bool(dagger)), int(precision), int(nrhs),
                                        ctypes.byref(comm)))


def qcd_slab_cg_solve(ctx, x_ptr, b_ptr, nrhs, params, stats, comm):
    s = lib().qcd_slab_cg_solve(ctx, x_ptr, b_ptr, int(nrhs), ctypes.byref(params), stats, ctypes.byref(comm))
    if s not in (QCD_OK, 6):
        _check(s)
    return s


def qcd_last_error():
    return lib().qcd_last_error().decode()


def solver_params(tol=1e-8, max_iter=20000, inner_prec=32, reliable_every=50, reliable_delta=0.1, use_x0=False):
    return SolverParams(float(tol), int(max_iter), int(inner_prec), int(reliable_every), float(reliable_delta),
                        int(bool(use_x0)))


# ---- torch-facing owner of a context ----------------------------------------------------------------------
def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class CloverWilson:
    """Owns one qcd_ctx for a lattice dims = (X, Y, Z, T) on the current CUDA device and stream."""

    def __init__(self, dims, t_bc=-1.0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libqcd needs a CUDA device")
        self.dims = tuple(int(d) for d in dims)
        X, Y, Z, T = self.dims
        self.V = X * Y * Z * T
        self.Vh = self.V // 2
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = qcd_create(self.dims, t_bc, ctypes.c_void_p(self.stream.cuda_stream))
        self.kappa = None
        self.csw = None

    def close(self):
        if self.ctx is not None:
            qcd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _spinor(self, t, nrhs=None):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("fields must be contiguous complex128 CUDA tensors")
        if t.numel() % (self.Vh * 12):
            raise ValueError("field size is not a multiple of V/2 * 12")
        return t.numel() // (self.Vh * 12)

    def load_gauge(self, U, recon12=False):
        """U: complex128 [T, Z, Y, X, 4, 3, 3] on the GPU (device copy) or on the CPU (host copy)."""
        if U.dtype != torch.complex128 or not U.is_contiguous() or U.numel() != self.V * 36:
            raise ValueError("U must be a contiguous complex128 tensor of V*4*9 elements")
        qcd_load_gauge(self.ctx, _ptr(U), U.is_cuda, QCD_GAUGE_RECON12 if recon12 else 0)

    def clover_build(self, kappa, csw):
        qcd_clover_build(self.ctx, kappa, csw)
        self.kappa, self.csw = float(kappa), float(csw)

    def dslash(self, x, op, dagger=False, precision=64):
        n = self._spinor(x)
        out = torch.empty_like(x)
        qcd_dslash(self.ctx, _ptr(out), _ptr(x), op, dagger, precision, n)
        return out

    def cg_solve(self, b, x0=None, **kw):
        """Solve Mhat^dag Mhat x = b; returns (x, [stats dict per RHS], converged)."""
        n = self._spinor(b)
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        prm = solver_params(use_x0=x0 is not None, **kw)
        st = (SolverStats * n)()
        s = qcd_cg_solve(self.ctx, _ptr(x), _ptr(b), n, prm, st)
        return x, [st[i].as_dict() for i in range(n)], s == QCD_OK

    def fermion_force(self, phi_or_x, input_is_solution=False, gradient=False, clover_det=False, **kw):
        """Force (or Wirtinger gradient) [T, Z, Y, X, 4, 3, 3] summed over the RHS of phi_or_x; with
        clover_det the force of S_det = -2 log det A_oo is added (phi_or_x may then be None: that
        term alone)."""
        n = 0 if phi_or_x is None else self._spinor(phi_or_x)
        X, Y, Z, T = self.dims
        F = torch.empty((T, Z, Y, X, 4, 3, 3), dtype=torch.complex128, device=self.device)
        flags = ((QCD_FORCE_INPUT_IS_SOLUTION if input_is_solution else 0) | (QCD_FORCE_GRADIENT if gradient else 0)
                 | (QCD_FORCE_CLOVER_DET if clover_det else 0))
        prm = None if (input_is_solution or n == 0) else solver_params(**kw)
        st = (SolverStats * max(n, 1))()
        qcd_fermion_force(self.ctx, _ptr(F), None if n == 0 else _ptr(phi_or_x), n, flags, prm, st)
        return F, [st[i].as_dict() for i in range(n)]

    def clover_logdet(self):
        """(sum_{x even}, sum_{x odd}) of log det A(x); the determinant term is S_det = -2 * [1]."""
        return qcd_clover_logdet(self.ctx)

    def prepare_source(self, b_e, b_o=None):
        """b_e + kappa D_eo A_oo^-1 b_o: the even source of the full-lattice system."""
        n = self._spinor(b_e)
        out = torch.empty_like(b_e)
        qcd_prepare_source(self.ctx, _ptr(out), _ptr(b_e), None if b_o is None else _ptr(b_o), n)
        return out

    def reconstruct_odd(self, x_e, b_o=None):
        """x_o = A_oo^-1 (b_o + kappa D_oe x_e): the odd half of the full-lattice solution."""
        n = self._spinor(x_e)
        out = torch.empty_like(x_e)
        qcd_reconstruct_odd(self.ctx, _ptr(out), _ptr(x_e), None if b_o is None else _ptr(b_o), n)
        return out

    def _links(self, t):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous() or t.numel() != self.V * 36:
            raise ValueError("link-shaped fields must be contiguous complex128 CUDA tensors of V*4*9 elements")

    def gauge_force(self, beta, gradient=False, out=None):
        """Wilson gauge force (or gradient) of the loaded links; added to `out` when given."""
        X, Y, Z, T = self.dims
        F = out if out is not None else torch.empty((T, Z, Y, X, 4, 3, 3), dtype=torch.complex128,
                                                     device=self.device)
        self._links(F)
        flags = (QCD_FORCE_GRADIENT if gradient else 0) | (QCD_FORCE_ACCUMULATE if out is not None else 0)
        qcd_gauge_force(self.ctx, _ptr(F), beta, flags)
        return F

    def plaquette(self):
        """Mean of Re tr P_{mu nu}(x) / 3 over sites and planes of the loaded links."""
        return qcd_plaquette(self.ctx)

    def kinetic_energy(self, P):
        self._links(P)
        return qcd_kinetic_energy(self.ctx, _ptr(P))

    def update_links(self, U, P, eps):
        """U <- exp(eps P) U (reunitarised), in place."""
        self._links(U)
        self._links(P)
        qcd_update_links(self.ctx, _ptr(U), _ptr(P), eps)
        return U

    def r_step(self, U, P, eta, eps, beta, clover_det=True, defer_clover=False, **kw):
        """One two-flavour R-algorithm step on U and P in place (noise eta [n, V/2, 4, 3] or None);
        defer_clover leaves the new links' clover term unbuilt (for the steps of a trajectory)."""
        self._links(U)
        self._links(P)
        n = 0 if eta is None else self._spinor(eta)
        st = (SolverStats * max(n, 1))()
        flags = (QCD_FORCE_CLOVER_DET if clover_det else 0) | (QCD_R_STEP_DEFER_CLOVER if defer_clover else 0)
        s = qcd_r_step(self.ctx, _ptr(U), _ptr(P), None if eta is None else _ptr(eta), n, eps, beta,
                       flags, solver_params(**kw) if n else None, st)
        return [st[i].as_dict() for i in range(n)], s == QCD_OK

    def polyakov(self):
        """Complex mean over spatial sites of tr prod_t U_t / 3 for the loaded links."""
        return qcd_polyakov(self.ctx)

    def pbp(self, eta_e, eta_o, **kw):
        """Stochastic psi-bar psi estimates Re eta^dag M^-1 eta / (2V), one per noise vector."""
        n = self._spinor(eta_e)
        if self._spinor(eta_o) != n:
            raise ValueError("eta_e and eta_o must hold the same number of fields")
        st = (SolverStats * n)()
        vals, s = qcd_pbp(self.ctx, _ptr(eta_e), _ptr(eta_o), n, solver_params(**kw), st)
        return vals, [st[i].as_dict() for i in range(n)], s == QCD_OK

    def profile(self, enable=True):
        qcd_profile(self.ctx, enable)

    def profile_read(self):
        return qcd_profile_read(self.ctx)


class CloverPseudofermionAction(torch.autograd.Function):
    """S(U, phi) = sum_i phi_i^dag (Mhat[U]^dag Mhat[U])^-1 phi_i and its gradients.

    forward(U, phi, op, kappa, csw, solver_kw, recompute): loads U into the
    CloverWilson context op, builds the clover term, solves (mixed or FP64
    precision per solver_kw) and returns S as a 0-d float64 tensor computed from
    the library's FP64 <phi, X>.  backward returns dS/dU as the Wirtinger
    gradient G = dS/dRe U + i dS/dIm U (torch's convention for a real loss of a
    complex input) from the library's force kernels, and dS/dphi = 2 X.  With
    recompute=True the solution X is not kept between forward and backward; the
    backward solves again.
    """

    @staticmethod
    def forward(ctx, U, phi, op, kappa, csw, solver_kw=None, recompute=False):
        solver_kw = dict(solver_kw or {})
        op.load_gauge(U.detach().contiguous(), recon12=solver_kw.pop("recon12", False))
        op.clover_build(kappa, csw)
        x, stats, ok = op.cg_solve(phi.detach().contiguous(), **solver_kw)
        if not ok:
            raise QCDError(6, "CG did not converge in the action's forward solve")
        S = sum(s["b_dot_x"] for s in stats)
        ctx.op = op
        ctx.solver_kw = solver_kw
        ctx.recompute = recompute
        ctx.kappa, ctx.csw = kappa, csw
        if recompute:
            ctx.save_for_backward(U, phi)
        else:
            ctx.save_for_backward(U, phi, x)
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, gS):
        op = ctx.op
        saved = ctx.saved_tensors
        U, phi = saved[0], saved[1]
        op.load_gauge(U.detach().contiguous())
        op.clover_build(ctx.kappa, ctx.csw)
        if ctx.recompute:
            x, _, ok = op.cg_solve(phi.detach().contiguous(), **ctx.solver_kw)
            if not ok:
                raise QCDError(6, "CG did not converge in the recomputation")
        else:
            x = saved[2]
        G, _ = op.fermion_force(x, input_is_solution=True, gradient=True)
        gU = gS * G if ctx.needs_input_grad[0] else None
        gphi = gS * 2.0 * x if ctx.needs_input_grad[1] else None
        return gU, gphi, None, None, None, None, None
