"""Time-slab decomposition of the operator and the CG solve over several GPUs (include/qcd.h,
qcd_create_slab and the qcd_slab_* calls): argument marshalling and the communication plumbing.

The paper runs its application as MPI processes that each hold part of the lattice and exchange
boundary data between kernels (Sec. 4).  Here rank r of W holds the time slices
t_offset .. t_offset + t_local - 1 of the global lattice.  Every hopping pass exchanges six complex
numbers per t-face site with the two neighbouring slabs, and every CG reduction is summed over the
ranks; the library asks for both through callbacks, which this module provides:

* ``TorchHaloComm`` -- torch.distributed (NCCL for CUDA tensors across processes, gloo for CPU
  tensors): paired sends and receives to the ranks below and above, and an all-reduce;
* ``NativeSlabGroup`` -- several slabs of one lattice in one process on one GPU, each driven by a host
  thread of its own; the library's in-process group (qcd_local_group_*) makes the exchanges and sums
  (halo kernels reading the neighbours' send buffers in place, ordered by CUDA events between the
  slabs' streams), with no Python in the loop;
* ``LocalSlabGroup`` -- the same with the exchanges and sums written in Python (torch copies after
  host synchronisation), a reference for the native group.

``SlabCloverWilson`` owns one slab context, its four halo buffers and the ctypes callbacks.  All
arithmetic runs in the library's kernels; this module only moves buffers between ranks.
"""

import ctypes
import threading

import numpy as np
import torch

from . import qcd as Q


# ---- layout helpers (no GPU) -----------------------------------------------------------------------------
def slab_bounds(T, world, rank):
    """(t_offset, t_local) of rank `rank` when T time slices are cut into `world` slabs of even thickness,
    as equal as the pairs of slices allow (earlier ranks take the extra pairs)."""
    if T % 2 or T < 2 * world:
        raise ValueError(f"T = {T} cannot be cut into {world} slabs of an even number of slices")
    pairs, extra = divmod(T // 2, world)
    t_local = 2 * (pairs + (1 if rank < extra else 0))
    t_offset = 2 * (rank * pairs + min(rank, extra))
    return t_offset, t_local


def extended_links(U, t_offset, t_local):
    """The links a slab context loads: global time slices t_offset-2 .. t_offset+t_local+1 (mod T) of the
    canonical gauge field U [T, Z, Y, X, 4, 3, 3] (numpy array or torch tensor)."""
    T = U.shape[0]
    idx = [(t_offset - 2 + k) % T for k in range(t_local + 4)]
    if isinstance(U, torch.Tensor):
        return U[torch.as_tensor(idx, device=U.device)].contiguous()
    return np.ascontiguousarray(U[idx])


def slab_rows(dims, t_offset, t_local):
    """The half-index range [start, stop) of a slab in a global even- or odd-site field [V/2, 4, 3]: the
    slab's time slices are contiguous in the lexicographic order and keep their parity (t_offset even)."""
    X, Y, Z, _ = dims
    half = X * Y * Z // 2
    return t_offset * half, (t_offset + t_local) * half


# ---- communication ---------------------------------------------------------------------------------------
class TorchHaloComm:
    """Halo exchange and sums over the ranks of a torch.distributed process group.  Rank r's slab has
    rank (r + 1) mod W above it and rank (r - 1) mod W below it (periodic in time)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.upper = (self.rank + 1) % self.world
        self.lower = (self.rank - 1) % self.world

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        """recv_hi <- the upper rank's send_lo; recv_lo <- the lower rank's send_hi."""
        if self.world == 1:
            recv_hi.copy_(send_lo)
            recv_lo.copy_(send_hi)
            return
        dist = self.dist
        up = dist.get_global_rank(self.group, self.upper) if self.group is not None else self.upper
        lo = dist.get_global_rank(self.group, self.lower) if self.group is not None else self.lower
        # the same order on every rank: with two ranks both neighbours are one process, and the
        # messages between a pair are matched in the order they are posted
        ops = [dist.P2POp(dist.isend, send_lo, lo, self.group), dist.P2POp(dist.isend, send_hi, up, self.group),
               dist.P2POp(dist.irecv, recv_hi, up, self.group), dist.P2POp(dist.irecv, recv_lo, lo, self.group)]
        for w in dist.batch_isend_irecv(ops):
            w.wait()

    def allreduce(self, values):
        if self.world > 1:
            self.dist.all_reduce(values, group=self.group)


class _CudaArray:
    """A device pointer seen as a torch tensor (through __cuda_array_interface__, no copy)."""

    def __init__(self, ptr, n, typestr="<f8"):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "strides": None}


def device_doubles(ptr, n):
    return torch.as_tensor(_CudaArray(ctypes.cast(ptr, ctypes.c_void_p).value, n), device="cuda")


class SlabCloverWilson:
    """Owns one slab context of a global lattice dims = (X, Y, Z, T) with its four halo buffers and the
    callbacks the qcd_slab_* calls make.  comm: a NativeSlabGroup member (the library's buffers and
    callbacks), or an object with exchange(send_lo, send_hi, recv_lo, recv_hi) (uint8 device tensors of
    the bytes to move) and allreduce(values) (a float64 device tensor): TorchHaloComm, or a
    LocalSlabGroup member."""

    def __init__(self, dims, t_offset, t_local, comm, t_bc=-1.0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("libqcd needs a CUDA device")
        self.dims = tuple(int(d) for d in dims)
        self.t_offset, self.t_local = int(t_offset), int(t_local)
        X, Y, Z, _ = self.dims
        self.local_dims = (X, Y, Z, self.t_local)
        self.Vh = X * Y * Z * self.t_local // 2
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = Q.qcd_create_slab(self.dims, self.t_offset, self.t_local, t_bc,
                                     ctypes.c_void_p(self.stream.cuda_stream))
        self.comm = comm
        self._errors = []
        if isinstance(comm, _NativeMember):
            # the group's buffers and native callbacks
            self.comm_struct = Q.qcd_local_group_join(comm.group.handle, comm.rank, self.ctx)
            self.bufs, self._fns = None, None
            return
        nbytes = Q.qcd_slab_halo_bytes(self.ctx, 64, 8)  # the largest: FP64 reliable updates of 8 RHS
        self.bufs = [torch.zeros(nbytes, dtype=torch.uint8, device="cuda") for _ in range(4)]

        def exchange(user, nb):
            try:
                with torch.cuda.stream(self.stream):
                    self.comm.exchange(*(b[:nb] for b in self.bufs))
                return 0
            except Exception as e:  # reported to the library as a failed callback
                self._errors.append(e)
                return 1

        def allreduce(user, values, n):
            try:
                with torch.cuda.stream(self.stream):
                    self.comm.allreduce(device_doubles(values, n))
                return 0
            except Exception as e:
                self._errors.append(e)
                return 1

        self._fns = (Q.EXCHANGE_FN(exchange), Q.ALLREDUCE_FN(allreduce))  # kept alive with the object
        self.comm_struct = Q.SlabComm(*(b.data_ptr() for b in self.bufs), self._fns[0], self._fns[1], None)

    def close(self):
        if self.ctx is not None:
            Q.qcd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _n(self, t):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous() or t.numel() % (self.Vh * 12):
            raise ValueError("slab fields must be contiguous complex128 CUDA tensors of nrhs x V_slab/2 x 12")
        return t.numel() // (self.Vh * 12)

    def load_gauge(self, U_ext, recon12=False):
        """U_ext: the extended links of this slab (extended_links), complex128 on the GPU or the CPU."""
        X, Y, Z, _ = self.dims
        if U_ext.dtype != torch.complex128 or not U_ext.is_contiguous() or \
                U_ext.numel() != (self.t_local + 4) * X * Y * Z * 36:
            raise ValueError("U_ext must be contiguous complex128 [t_local + 4, Z, Y, X, 4, 3, 3]")
        Q.qcd_load_gauge(self.ctx, Q._ptr(U_ext), U_ext.is_cuda, Q.QCD_GAUGE_RECON12 if recon12 else 0)

    def clover_build(self, kappa, csw):
        Q.qcd_clover_build(self.ctx, kappa, csw)

    def clover_logdet(self):
        return Q.qcd_clover_logdet(self.ctx)

    def dslash(self, x, op, dagger=False, precision=64):
        n = self._n(x)
        out = torch.empty_like(x)
        Q.qcd_slab_dslash(self.ctx, Q._ptr(out), Q._ptr(x), op, dagger, precision, n, self.comm_struct)
        return out

    def cg_solve(self, b, x0=None, **kw):
        """Mhat^dag Mhat x = b on the whole lattice, this rank holding its slab of b and x; returns (x,
        [stats per RHS], converged)."""
        n = self._n(b)
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        prm = Q.solver_params(use_x0=x0 is not None, **kw)
        st = (Q.SolverStats * n)()
        s = Q.qcd_slab_cg_solve(self.ctx, Q._ptr(x), Q._ptr(b), n, prm, st, self.comm_struct)
        return x, [st[i].as_dict() for i in range(n)], s == Q.QCD_OK


def _run_threads(n, fns, abort):
    """Call fns[r]() on thread r; returns their results (re-raises the first error after abort())."""
    out = [None] * n
    errs = []

    def body(r):
        try:
            out[r] = fns[r]()
        except BaseException as e:
            errs.append(e)
            abort()

    th = [threading.Thread(target=body, args=(r,)) for r in range(n)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    return out


class NativeSlabGroup:
    """Several slabs of one lattice in this process, all on one GPU: member(r) is the comm of slab r,
    whose exchanges and sums the library's in-process group makes (qcd_local_group_*: CUDA events
    between the slabs' streams, one host barrier per exchange or sum only to publish them, halos read
    in place from the neighbours' send buffers, sums in slab order).  Each
    slab's calls must run on a host thread of their own (run()); ctypes releases the interpreter lock
    during the calls, so the slabs' threads run side by side.  close() after the slabs' last call."""

    def __init__(self, n):
        self.n = n
        self.handle = Q.qcd_local_group_create(n)

    def member(self, rank):
        return _NativeMember(self, rank)

    def run(self, fns):
        return _run_threads(self.n, fns, lambda: Q.qcd_local_group_abort(self.handle))

    def close(self):
        if self.handle is not None:
            Q.qcd_local_group_destroy(self.handle)
            self.handle = None


class _NativeMember:
    def __init__(self, group, rank):
        self.group = group
        self.rank = rank


class LocalSlabGroup:
    """Several slabs of one lattice in this process (for example all on one GPU): member(r) is the comm
    object of slab r; each slab's calls must run on a host thread of their own (run()).  An exchange or a
    sum waits for every slab at a host barrier, then copies between the slabs' buffers on the calling
    slab's stream; the sums are added in slab order, so every slab gets the same bits."""

    def __init__(self, n):
        self.n = n
        self.barrier = threading.Barrier(n)
        self.halo = [None] * n
        self.values = [None] * n
        self.streams = [None] * n

    def member(self, rank):
        return _LocalMember(self, rank)

    def run(self, fns):
        """Call fns[r]() on thread r for every slab; returns their results (re-raises the first error)."""
        return _run_threads(self.n, fns, self.barrier.abort)


class _LocalMember:
    def __init__(self, group, rank):
        self.g = group
        self.rank = rank

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        g, r = self.g, self.rank
        stream = torch.cuda.current_stream()
        stream.synchronize()            # this slab's faces are packed
        g.halo[r] = (send_lo, send_hi)
        g.barrier.wait()                # every slab's are
        recv_hi.copy_(g.halo[(r + 1) % g.n][0])
        recv_lo.copy_(g.halo[(r - 1) % g.n][1])
        stream.synchronize()            # this slab has read its neighbours' faces
        g.barrier.wait()                # every slab has, before any packs again

    def allreduce(self, values):
        g, r = self.g, self.rank
        stream = torch.cuda.current_stream()
        g.values[r] = values.cpu()      # synchronises this slab's stream
        g.barrier.wait()
        total = g.values[0].clone()
        for k in range(1, g.n):
            total += g.values[k]
        values.copy_(total.to(values.device))
        stream.synchronize()
        g.barrier.wait()
