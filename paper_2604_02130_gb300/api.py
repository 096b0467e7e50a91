"""Python binding of the C ABI (include/fd.h).  Marshalling only: every step of the
computation runs in libfd.so's CUDA kernels; torch provides device memory and streams.

    ctx = Context(0)
    batch = Batch(ctx, [(E, Einv, phi, n_stab), ...], want="force", prec="fp64")
    out = batch.run()            # enqueues on the current torch stream
    out.logdet, out.G, out.F     # complex128 tensors on the device
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import torch

from . import _lib as L


class FdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("fd error %d: %s" % (code, msg))
        self.code = code


def _stream_ptr(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """Owns an fd_ctx (workspace, descriptor tables) on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = L.load()
        if not torch.cuda.is_available():
            raise RuntimeError("fd requires a CUDA device (there is no CPU path)")
        torch.cuda.set_device(device)
        self.device = device
        h = ctypes.c_void_p()
        rc = self.lib.fd_ctx_create(ctypes.byref(h), device)
        if rc != L.FD_OK:
            raise FdError(rc, "fd_ctx_create failed")
        self.h = h

    def check(self, rc: int):
        if rc != L.FD_OK:
            raise FdError(rc, self.lib.fd_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.fd_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, batch: int, stream=None) -> List[int]:
        arr = (ctypes.c_int * max(1, batch))()
        self.lib.fd_status(self.h, _stream_ptr(stream), arr, batch)
        return [arr[i] for i in range(batch)]

    def debug_skip_chains(self, on: bool):
        """Failure-detection test hook (fd_debug_skip_chains): phased calls skip their chain
        launch, so the dependent tasks' bounded waits run out and report FD_ERR_TIMEOUT."""
        self.check(self.lib.fd_debug_skip_chains(self.h, 1 if on else 0))

    def set_force_split(self, mode: int) -> None:
        """Time-parallel force chains (fd_set_force_split): -1 automatic (halves for FP64
        calls with 4 * batch <= SMs, segments for long chains of the mixed path), 0 never,
        1 wherever the configuration has enough blocks."""
        self.check(self.lib.fd_set_force_split(self.h, int(mode)))

    def last_launch_count(self) -> int:
        return self.lib.fd_last_launch_count(self.h)

    def set_timing(self, on: bool):
        self.check(self.lib.fd_set_timing(self.h, 1 if on else 0))

    def last_kernel_ms(self, max_launches: int = 64) -> List[float]:
        arr = (ctypes.c_double * max_launches)()
        n = self.lib.fd_last_kernel_ms(self.h, arr, max_launches)
        if n < 0:
            self.check(n)
        return [arr[i] for i in range(n)]

    def tune_nstab(self, problem: Tuple, candidates: Sequence[int], rel_budget: float,
                   prec: str = "3xtf32", stats: bool = False):
        """The fastest QR interval among candidates whose log det and G stay within rel_budget of
        FP64 (fd_tune_nstab_stats); 0 if none does.  With stats, also returns each candidate's
        error and time: (best, [err], [ms])."""
        E, Einv, phi, _ = problem
        p = L.fd_problem(phi.shape[1], phi.shape[0], int(candidates[0]), 0, E.data_ptr(),
                         Einv.data_ptr() if Einv is not None else None, phi.data_ptr())
        cand = (ctypes.c_int * len(candidates))(*candidates)
        best = ctypes.c_int()
        err = (ctypes.c_double * len(candidates))()
        ms = (ctypes.c_double * len(candidates))()
        self.check(self.lib.fd_tune_nstab_stats(self.h, ctypes.byref(p), cand, len(candidates),
                                                rel_budget, L.PRECISIONS[prec],
                                                ctypes.byref(best), err, ms))
        if stats:
            return best.value, list(err), list(ms)
        return best.value

    def tune_save(self, path: str):
        self.check(self.lib.fd_tune_save(self.h, path.encode()))

    def tune_load(self, path: str) -> int:
        n = self.lib.fd_tune_load(self.h, path.encode())
        if n < 0:
            self.check(n)
        return n

    def measure_fp64_issue(self) -> List[float]:
        """Cycles per FP64 instruction: [1 lane, 32 lanes, 1 of 8 busy warps]."""
        arr = (ctypes.c_double * 3)()
        self.check(self.lib.fd_measure_fp64_issue(self.h, arr))
        return [arr[0], arr[1], arr[2]]

    def measure_fp64_peak(self) -> float:
        g = ctypes.c_double()
        self.check(self.lib.fd_measure_fp64_peak(self.h, ctypes.byref(g)))
        return g.value


@dataclass
class Result:
    logdet: torch.Tensor  # (batch,) complex128
    G: Optional[List[torch.Tensor]]  # nx x nx complex128 each
    F: Optional[List[torch.Tensor]]  # nt x nx complex128 each
    Gtau: Optional[List[torch.Tensor]] = None  # nt x nx x nx complex128 each: G(tau, 0)
    nferm: Optional[torch.Tensor] = None  # (batch,) complex128: 1 - tr G / nx
    R: Optional[List[torch.Tensor]] = None  # (nt,) complex128 each: tr(O G_r)


class Batch:
    """A fixed batch of configurations with preallocated outputs; run() enqueues one call.

    problems: sequence of (E, Einv, phi, n_stab) with E, Einv (nx, nx) float64 and phi (nt, nx)
    float64 CUDA tensors (Einv may be None unless F, G(tau, 0) or R is wanted).

    want: "logdet", or "+"-joined outputs among "green" (G), "force" (F), "gtau" (the
    unequal-time G(tau, 0), tau = 0..nt-1), "nferm" (fermion number 1 - tr G / nx) and
    "response" (R[r] = tr(O G_r) for the per-configuration operators `operators`, (nx, nx)
    float64 CUDA tensors); log det always comes along.  "gtau" does not combine with "nferm" or
    "response"."""

    WANT_BITS = {"logdet": 1, "green": 2, "force": 4, "gtau": 8, "response": 16, "nferm": 32}

    def __init__(self, ctx: Context, problems: Sequence[Tuple], want: str = "logdet",
                 prec: str = "fp64", operators: Optional[Sequence[torch.Tensor]] = None):
        parts = set(want.split("+"))
        if not parts or not parts <= set(self.WANT_BITS):
            raise ValueError(want)
        if "gtau" in parts and parts & {"nferm", "response"}:
            raise ValueError("gtau does not combine with nferm/response")
        if ("response" in parts) != (operators is not None):
            raise ValueError("want 'response' needs operators (and only then)")
        self.ctx = ctx
        self.want = want
        self.what = 1
        for p in parts:
            self.what |= self.WANT_BITS[p]
        self.prec = L.PRECISIONS[prec]
        self.n = len(problems)
        self._keep = []
        arr = (L.fd_problem * max(1, self.n))()
        dev = torch.device("cuda", ctx.device)
        for c, (E, Einv, phi, n_stab) in enumerate(problems):
            for t in (E, phi) + ((Einv,) if Einv is not None else ()):
                if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                    raise ValueError("inputs must be contiguous float64 CUDA tensors")
            nt, nx = phi.shape
            arr[c].nx, arr[c].nt, arr[c].n_stab, arr[c].reserved = nx, nt, int(n_stab), 0
            arr[c].expA = E.data_ptr()
            arr[c].expA_inv = Einv.data_ptr() if Einv is not None else None
            arr[c].phi = phi.data_ptr()
            self._keep += [E, Einv, phi]
        self.problems = arr
        self.logdet_buf = torch.empty((self.n, 2), dtype=torch.float64, device=dev)
        self.G = None
        self.F = None
        self.Gtau = None
        self._Gp = None
        self._Fp = None
        self._Gtp = None
        # outputs live in one flat buffer each (one host copy fetches them all)
        self.G_flat = None
        self.F_flat = None
        self.Gtau_flat = None
        self.nferm_buf = None
        self.R = None
        self.R_flat = None
        self._Op = None
        self._Rp = None
        if self.what & 32:
            self.nferm_buf = torch.empty((self.n, 2), dtype=torch.float64, device=dev)
        if self.what & 16:
            if len(operators) != self.n:
                raise ValueError("one operator per configuration")
            for c, O in enumerate(operators):
                if not (O.is_cuda and O.dtype == torch.float64 and O.is_contiguous()
                        and tuple(O.shape) == (arr[c].nx, arr[c].nx)):
                    raise ValueError("operators must be contiguous (nx, nx) float64 CUDA tensors")
            self._keep += list(operators)
            self._Op = (ctypes.c_void_p * self.n)(*[O.data_ptr() for O in operators])
            self.R_flat, self.R = self._flat(dev, [(p.nt,) for p in arr[:self.n]])
            self._Rp = (ctypes.c_void_p * self.n)(*[r.data_ptr() for r in self.R])
        if self.what & 2:
            self.G_flat, self.G = self._flat(dev, [(p.nx, p.nx) for p in arr[:self.n]])
            self._Gp = (ctypes.c_void_p * self.n)(*[g.data_ptr() for g in self.G])
        if self.what & 4:
            self.F_flat, self.F = self._flat(dev, [(p.nt, p.nx) for p in arr[:self.n]])
            self._Fp = (ctypes.c_void_p * self.n)(*[f.data_ptr() for f in self.F])
        if self.what & 8:
            self.Gtau_flat, self.Gtau = self._flat(
                dev, [(p.nt, p.nx, p.nx) for p in arr[:self.n]])
            self._Gtp = (ctypes.c_void_p * self.n)(*[g.data_ptr() for g in self.Gtau])

    @staticmethod
    def _flat(dev, shapes):
        sizes = [math.prod(s) for s in shapes]
        flat = torch.empty(max(1, sum(sizes)), dtype=torch.complex128, device=dev)
        views, o = [], 0
        for s, k in zip(shapes, sizes):
            views.append(flat[o:o + k].view(*s))
            o += k
        return flat, views

    def plan(self) -> List[dict]:
        """The launch plan of this batch (one dict per size class), see fd_plan_query."""
        info = (ctypes.c_int * (8 * 64))()
        n = self.ctx.lib.fd_plan_query(self.ctx.h, self.n, self.problems, self.what & 31,
                                       self.prec, info, 64)
        if n < 0:
            self.ctx.check(n)
        keys = ("nx", "kernel", "threads", "smem", "grid", "ctas_per_sm", "scratch_kib", "configs")
        return [dict(zip(keys, info[8 * g:8 * g + 8])) for g in range(min(n, 64))]

    def reserve(self):
        self.ctx.check(self.ctx.lib.fd_reserve(self.ctx.h, self.n, self.problems,
                                               self.what & 31, self.prec))

    def run(self, stream=None) -> Result:
        lib, h = self.ctx.lib, self.ctx.h
        s = _stream_ptr(stream)
        ld = ctypes.c_void_p(self.logdet_buf.data_ptr())
        if self.what & 8:
            rc = lib.fd_green_tau(h, self.n, self.problems, ld, self._Gp, self._Gtp, self._Fp,
                                  self.prec, s)
        elif self.what & (16 | 32):
            nf = ctypes.c_void_p(self.nferm_buf.data_ptr()) if self.nferm_buf is not None else None
            rc = lib.fd_observables(h, self.n, self.problems, ld, self._Gp, self._Fp, nf,
                                    self._Op, self._Rp, self.prec, s)
        elif self.what & 4:
            rc = lib.fd_force(h, self.n, self.problems, ld, self._Gp, self._Fp, self.prec, s)
        elif self.what & 2:
            rc = lib.fd_green(h, self.n, self.problems, ld, self._Gp, self.prec, s)
        else:
            rc = lib.fd_logdet(h, self.n, self.problems, ld, self.prec, s)
        self.ctx.check(rc)
        nf = torch.view_as_complex(self.nferm_buf) if self.nferm_buf is not None else None
        return Result(torch.view_as_complex(self.logdet_buf), self.G, self.F, self.Gtau, nf,
                      self.R)

    def status(self, stream=None) -> List[int]:
        return self.ctx.status(self.n, stream)

    def tune(self, reps: int = 2):
        """Time 128 vs 256 threads per CTA for every size class of this batch (fd_tune)."""
        self.ctx.check(self.ctx.lib.fd_tune(self.ctx.h, self.n, self.problems, self.what & 31,
                                            self.prec, reps))

    def graph(self) -> "BatchGraph":
        """Capture this batch's call into a CUDA graph (fd_graph_create)."""
        return BatchGraph(self)


class BatchGraph:
    """A captured fd_* call over a Batch; launch() replays it with one cudaGraphLaunch.
    Inputs are read and outputs written through the Batch's tensors (update phi in place)."""

    def __init__(self, batch: Batch):
        if batch.what & (8 | 16 | 32):
            raise ValueError("G(tau, 0) and observables are not available through CUDA graphs")
        self.batch = batch
        ctx = batch.ctx
        h = ctypes.c_void_p()
        ld = ctypes.c_void_p(batch.logdet_buf.data_ptr())
        F = batch._Fp if batch.what & 4 else None
        ctx.check(ctx.lib.fd_graph_create(ctx.h, batch.n, batch.problems, ld, batch._Gp, F,
                                          batch.prec, ctypes.byref(h)))
        self.h = h

    def launch(self, stream=None) -> Result:
        ctx = self.batch.ctx
        ctx.check(ctx.lib.fd_graph_launch(ctx.h, self.h, _stream_ptr(stream)))
        b = self.batch
        return Result(torch.view_as_complex(b.logdet_buf), b.G, b.F)

    def status(self, stream=None) -> List[int]:
        return self.batch.ctx.status(self.batch.n, stream)

    def close(self):
        if getattr(self, "h", None):
            self.batch.ctx.lib.fd_graph_destroy(self.batch.ctx.h, self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx: Optional[Context] = None


def default_context() -> Context:
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context(torch.cuda.current_device())
    return _default_ctx


def logdet(problems, prec: str = "fp64", ctx: Optional[Context] = None) -> torch.Tensor:
    """log det(1 + B_Nt...B_1) for a batch, complex128 (batch,)."""
    return Batch(ctx or default_context(), problems, "logdet", prec).run().logdet.clone()


def green(problems, prec: str = "fp64", ctx: Optional[Context] = None):
    r = Batch(ctx or default_context(), problems, "green", prec).run()
    return r.logdet.clone(), r.G


def force(problems, prec: str = "fp64", with_green: bool = False,
          ctx: Optional[Context] = None):
    r = Batch(ctx or default_context(), problems, "force+green" if with_green else "force",
              prec).run()
    return r.logdet.clone(), r.G, r.F


def green_tau(problems, prec: str = "fp64", with_green: bool = False,
              with_force: bool = False, ctx: Optional[Context] = None):
    """log det and the unequal-time Green's function G(tau, 0), tau = 0..nt-1 (Section 4.2);
    returns (logdet, G or None, F or None, [Gtau (nt, nx, nx) per configuration])."""
    want = "+".join(["gtau"] + (["green"] if with_green else []) +
                    (["force"] if with_force else []))
    r = Batch(ctx or default_context(), problems, want, prec).run()
    return r.logdet.clone(), r.G, r.F, r.Gtau


def observables(problems, operators=None, prec: str = "fp64", with_force: bool = False,
                ctx: Optional[Context] = None):
    """log det, the fermion number 1 - tr G / nx (Section 4.1) and, with `operators` (one
    (nx, nx) float64 CUDA tensor per configuration), the response traces tr(O G_r) at every
    time slice; returns (logdet, nferm, [R (nt,)] or None, [F] or None)."""
    want = "+".join(["nferm"] + (["response"] if operators is not None else []) +
                    (["force"] if with_force else []))
    r = Batch(ctx or default_context(), problems, want, prec, operators).run()
    return r.logdet.clone(), r.nferm.clone(), r.R, r.F


def taylor_factors(n: int) -> List[complex]:
    """The product-form factors gamma_k fd_green_sparse uses for n factors (fd_taylor_factors):
    prod_k (1 + gamma_k x) = sum_{j<=n} x^j / j!."""
    lib = L.load()
    arr = (ctypes.c_double * 16)()
    rc = lib.fd_taylor_factors(int(n), arr)
    if rc != L.FD_OK:
        raise FdError(rc, "fd_taylor_factors(%d)" % n)
    return [complex(arr[2 * k], arr[2 * k + 1]) for k in range(n)]


def green_sparse(problems, hops, nfac: int = 4, with_green: bool = True,
                 ctx: Optional[Context] = None, stream=None):
    """Intermediate-volume variant (Sections 8-9; fd_green_sparse): log det and optionally G with
    every slice applied as prod_k (1 + gamma_k K) diag(e^{i phi_t}), K sparse.

    problems: sequence of (phi (nt, nx) float64, n_stab); hops: sequence of (col (nx, q) int32,
    val (nx, q) float64), the entries of K row by row (fd_inputs.sparse_rows); CUDA tensors.
    Returns (logdet (batch,) complex128, [G (nx, nx) complex128] or None)."""
    ctx = ctx or default_context()
    n = len(problems)
    if len(hops) != n:
        raise ValueError("one hopping table per configuration")
    dev = torch.device("cuda", ctx.device)
    arr = (L.fd_problem * max(1, n))()
    hop = (L.fd_sparse_hop * max(1, n))()
    for c, ((phi, n_stab), (col, val)) in enumerate(zip(problems, hops)):
        if not (phi.is_cuda and phi.dtype == torch.float64 and phi.is_contiguous()):
            raise ValueError("phi must be a contiguous float64 CUDA tensor")
        nt, nx = phi.shape
        if not (col.is_cuda and col.dtype == torch.int32 and col.is_contiguous()
                and col.dim() == 2 and col.shape[0] == nx):
            raise ValueError("col must be a contiguous (nx, q) int32 CUDA tensor")
        if not (val.is_cuda and val.dtype == torch.float64 and val.is_contiguous()
                and tuple(val.shape) == tuple(col.shape)):
            raise ValueError("val must be a contiguous float64 CUDA tensor shaped like col")
        arr[c].nx, arr[c].nt, arr[c].n_stab, arr[c].reserved = nx, nt, int(n_stab), 0
        arr[c].expA = None
        arr[c].expA_inv = None
        arr[c].phi = phi.data_ptr()
        hop[c].q, hop[c].nfac = int(col.shape[1]), int(nfac)
        hop[c].col, hop[c].val = col.data_ptr(), val.data_ptr()
    logdet = torch.empty((max(1, n), 2), dtype=torch.float64, device=dev)
    G = None
    Gp = None
    if with_green:
        G = [torch.empty((p[0].shape[1], p[0].shape[1]), dtype=torch.complex128, device=dev)
             for p in problems]
        Gp = (ctypes.c_void_p * max(1, n))(*[g.data_ptr() for g in G])
    ctx.check(ctx.lib.fd_green_sparse(ctx.h, n, arr, hop, ctypes.c_void_p(logdet.data_ptr()),
                                      Gp, _stream_ptr(stream)))
    return torch.view_as_complex(logdet)[:n], G


class BssSlices:
    """A prepared local-update call (fd_bss_update, Section 3) over fixed device buffers.

    The table of pointers is built once, so repeated calls -- a sweep over slices, or repeated
    hits on one slice with new proposals written into the same buffers -- cost one C call each.
    Per configuration: G (nx, nx) complex128 = G_{t-1} of the current field (updated in place),
    phi_rows (nx,) float64 = the field of slice t (updated in place), dphi/u/w (nx,) float64,
    accepted (nx,) int32 (written; allocated when not given).  run() returns the change of log
    det as a (batch,) complex128 view of a buffer that the next run overwrites."""

    def __init__(self, G: Sequence[torch.Tensor], phi_rows: Sequence[torch.Tensor],
                 dphi: Sequence[torch.Tensor], u: Sequence[torch.Tensor],
                 w: Sequence[torch.Tensor], accepted: Optional[Sequence[torch.Tensor]] = None,
                 ctx: Optional[Context] = None):
        self.ctx = ctx or default_context()
        self.n = n = len(G)
        dev = torch.device("cuda", self.ctx.device)
        self.arr = (L.fd_bss_slice * max(1, n))()
        self.accepted = []
        for c in range(n):
            nx = G[c].shape[0]
            if not (G[c].is_cuda and G[c].dtype == torch.complex128 and G[c].is_contiguous()
                    and tuple(G[c].shape) == (nx, nx)):
                raise ValueError("G must be contiguous (nx, nx) complex128 CUDA tensors")
            for t in (phi_rows[c], dphi[c], u[c], w[c]):
                if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                        and t.numel() == nx):
                    raise ValueError("phi_rows, dphi, u, w must be contiguous (nx,) float64 CUDA "
                                     "tensors")
            a = torch.empty(nx, dtype=torch.int32, device=dev) if accepted is None \
                else accepted[c]
            if not (a.is_cuda and a.dtype == torch.int32 and a.is_contiguous()
                    and a.numel() == nx):
                raise ValueError("accepted must be contiguous (nx,) int32 CUDA tensors")
            self.accepted.append(a)
            self.arr[c].nx, self.arr[c].reserved = nx, 0
            self.arr[c].G, self.arr[c].phi_row = G[c].data_ptr(), phi_rows[c].data_ptr()
            self.arr[c].dphi, self.arr[c].u = dphi[c].data_ptr(), u[c].data_ptr()
            self.arr[c].w, self.arr[c].accepted = w[c].data_ptr(), a.data_ptr()
        # the tensors stay referenced for as long as the table points at them
        self._keep = (list(G), list(phi_rows), list(dphi), list(u), list(w))
        self.out = torch.empty((max(1, n), 2), dtype=torch.float64, device=dev)

    def run(self, stream=None) -> torch.Tensor:
        self.ctx.check(self.ctx.lib.fd_bss_update(self.ctx.h, self.n, self.arr,
                                                  ctypes.c_void_p(self.out.data_ptr()),
                                                  _stream_ptr(stream)))
        return torch.view_as_complex(self.out)[:self.n]


def bss_update(G: Sequence[torch.Tensor], phi_rows: Sequence[torch.Tensor],
               dphi: Sequence[torch.Tensor], u: Sequence[torch.Tensor],
               w: Sequence[torch.Tensor], ctx: Optional[Context] = None, stream=None):
    """Local (BSS) updates at one time slice for a batch (Section 3; fd_bss_update), one call.

    Arguments as for BssSlices.  Returns (dlogdet (batch,) complex128: change of log det,
    [accepted (nx,) int32])."""
    s = BssSlices(G, phi_rows, dphi, u, w, ctx=ctx)
    return s.run(stream).clone(), s.accepted


class FermionLogDet(torch.autograd.Function):
    """log det(1 + B_Nt...B_1) as a differentiable function of the field phi, for one
    configuration (phi of shape (nt, nx), complex128 scalar out) or a batch sharing E
    (phi of shape (batch, nt, nx), (batch,) out).

    forward(phi, E, Einv, n_stab, prec) runs fd_logdet only: no checkpoints are kept.  The
    backward pass runs the adjoint force sweep (fd_force), which recomputes the stabilised
    checkpoints every n_stab slices from the field instead of storing partial products, and
    returns torch's gradient for a real input, grad_phi = Re(conj(grad_out) * F) with
    F = d logdet / d phi (Section 4, Eq. response_result).  A forward under torch.no_grad(), or
    with a phi that does not require a gradient, therefore costs one log det call."""

    @staticmethod
    def _problems(phi, E, Einv, n_stab):
        phis = phi.detach()
        phis = (phis if phis.dim() == 3 else phis.unsqueeze(0)).contiguous()
        return phis, [(E, Einv, phis[k], n_stab) for k in range(phis.shape[0])]

    @staticmethod
    def forward(ctx_, phi, E, Einv, n_stab, prec="fp64"):
        if phi.dim() not in (2, 3):
            raise ValueError("phi must be (nt, nx) or (batch, nt, nx)")
        c = default_context()
        phis, probs = FermionLogDet._problems(phi, E, Einv, n_stab)
        r = Batch(c, probs, "logdet", prec).run()
        ctx_.save_for_backward(phis)
        ctx_.E, ctx_.Einv, ctx_.n_stab, ctx_.prec = E, Einv, n_stab, prec
        ctx_.batched = phi.dim() == 3
        out = r.logdet.clone()
        return out if ctx_.batched else out[0]

    @staticmethod
    def backward(ctx_, grad_out):
        (phis,) = ctx_.saved_tensors
        if ctx_.Einv is None:
            raise ValueError("the gradient needs E^{-1} (Einv)")
        probs = [(ctx_.E, ctx_.Einv, phis[k], ctx_.n_stab) for k in range(phis.shape[0])]
        r = Batch(default_context(), probs, "force", ctx_.prec).run()
        F = torch.stack(r.F)
        g = grad_out if ctx_.batched else grad_out.reshape(1)
        grad = (g.conj().view(-1, 1, 1) * F).real
        return (grad if ctx_.batched else grad[0]), None, None, None, None
