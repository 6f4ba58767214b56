"""Python binding of libsp2.so: the C entry points under the same names.

Argument marshalling only. Every step of the SP2 path runs in the library's
CUDA kernels; this module turns torch tensors (device buffers) or numpy
arrays (host buffers, staged by the library) into pointers and sizes, and
allocates outputs of the matching kind. PyTorch provides device memory and the
current stream.

Functions (see include/sp2.h for the exact semantics):
  sp2_density(H, nocc, ...)                     Eq. DM0               -> (D, info)
  sp2_response(H, nocc, H1, ...)                Eq. DMPert (DM1)      -> (D1, D, info)
  sp2_susceptibility(H, nocc, A, direction=...) Eq. DMSuscept / DM2   -> (chi, D, info)
  sp2_adjoint(G, handle)                        Eq. DM2 on kept X_n   -> grad
  synchronize(handle)                           sp2_synchronize       -> info of the last call
  sp2_fermi(H, mu, kT, B, ...)                  Sec. V.B finite T     -> (D1, D, info)
  sp2_scf_response(H, nocc, norb, K, Vext, ...) Eq. DM_CP_SCF         -> (q, residuals, iters, traj)
  mlp_forward / mlp_loss_grad / mlp_train       learned SCF preconditioner
  response_contract(P, Q, diag_only=...)        Tr[P_l Q_k]           -> (L, K) float64
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

__all__ = ["Handle", "make_opts", "synchronize", "sp2_density", "sp2_response", "sp2_susceptibility",
           "sp2_adjoint", "sp2_fermi", "sp2_nonorth_susceptibility", "sp2_scf_response",
           "mlp_forward", "mlp_loss_grad",
           "mlp_train", "response_contract", "SP2Error"]

SP2Error = L.SP2Error


def make_opts(mode: str | int = "bf16x2", idem_tol: float = 0.0, floor_gate: float = -1.0,
              max_iter: int = 0, min_iter: int = -1, sigma=None, bounds=None,
              ckpt_k: int | str = 0, keep_history: bool = False, time_kernels: bool = False,
              tail_f: float = 0.0, block_tau: float | None = None):
    """sp2_opts with the library defaults for everything not given. Returns
    (opts, keepalive) where keepalive holds the branch array referenced by
    opts.sigma_in. ckpt_k="auto" selects SP2_CKPT_AUTO (keep as much of the
    X_n history as device memory holds). block_tau (not None): the
    thresholded block-sparse recursion with that block threshold
    (sp2_density only)."""
    lib = L.load()
    o = L.Opts()
    lib.sp2_default_opts(C.byref(o))
    o.mode = L.MODES[mode] if isinstance(mode, str) else int(mode)
    o.idem_tol = float(idem_tol)
    o.floor_gate = float(floor_gate)
    o.max_iter = int(max_iter)
    o.min_iter = int(min_iter)
    o.ckpt_k = L.CKPT_AUTO if ckpt_k == "auto" else int(ckpt_k)
    o.keep_history = 1 if keep_history else 0
    o.time_kernels = 1 if time_kernels else 0
    o.tail_f = float(tail_f)
    if block_tau is not None:
        o.block_sparse = 1
        o.block_tau = float(block_tau)
    keep = None
    if sigma is not None:
        arr = (C.c_int8 * max(1, len(sigma)))(*[int(s) for s in sigma])
        o.fixed_m = len(sigma)
        o.sigma_in = C.cast(arr, C.POINTER(C.c_int8))
        keep = arr
    if bounds is not None:
        o.eps_min, o.eps_max = float(bounds[0]), float(bounds[1])
    return o, keep


def _dtype_code(x) -> int:
    dt = x.dtype
    if dt in (torch.float64, np.float64):
        return L.F64
    if dt in (torch.float32, np.float32):
        return L.F32
    raise TypeError(f"unsupported element type {dt}: float64 or float32 expected")


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        if not x.is_cuda:
            raise ValueError("torch tensors must live on a CUDA device (use numpy arrays for host buffers)")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"expected a torch.Tensor or numpy.ndarray, got {type(x)}")


def _empty_like(x, shape):
    if isinstance(x, torch.Tensor):
        return torch.empty(shape, dtype=x.dtype, device=x.device)
    return np.empty(shape, dtype=x.dtype)


class Handle:
    """Owns an sp2 handle (workspace, kept X_n history) on the current device."""

    def __init__(self, workspace_limit: int = 0):
        self.lib = L.load()
        self.h = C.c_void_p()
        stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
        rc = self.lib.sp2_create(C.byref(self.h), C.c_void_p(stream), C.c_size_t(workspace_limit))
        if rc != L.OK:
            raise L.SP2Error(rc, "sp2_create failed (no usable CUDA device?)")

    def bind_stream(self):
        if torch.cuda.is_available():
            self.lib.sp2_set_stream(self.h, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    def check(self, rc: int, allow_noconv: bool = False):
        if rc == L.OK or (allow_noconv and rc == L.ENOCONV):
            return
        raise L.SP2Error(rc, self.lib.sp2_last_error(self.h).decode())

    def set_option(self, option: str, value: int):
        """Product-kernel launch settings (sp2_set_option): "wait_limit_ns",
        "withhold_load" (test hook of the timed-out wait path), "fused_response" or
        "pair_tiles"."""
        code = {"wait_limit_ns": L.OPTION_WAIT_LIMIT_NS, "withhold_load": L.OPTION_WITHHOLD_LOAD,
                "fused_response": L.OPTION_FUSED_RESPONSE, "pair_tiles": L.OPTION_PAIR_TILES}[option]
        self.check(self.lib.sp2_set_option(self.h, code, int(value)))

    def workspace_bytes(self) -> int:
        return int(self.lib.sp2_workspace_bytes(self.h))

    def release_history(self):
        self.lib.sp2_release_history(self.h)

    def close(self):
        if self.h:
            self.lib.sp2_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default: dict = {}


def default_handle() -> Handle:
    dev = torch.cuda.current_device() if torch.cuda.is_available() else -1
    h = _default.get(dev)
    if h is None:
        h = Handle()
        _default[dev] = h
    return h


def _info_arg(sync: bool):
    """The info struct of a call, or None for a call that returns without waiting
    (complete it with synchronize(handle))."""
    return L.Info() if sync else None


def _info_ref(info):
    return C.byref(info) if info is not None else None


def _info_dict(info):
    return info.to_dict() if info is not None else None


def synchronize(handle: Handle | None = None, allow_noconv: bool = False) -> dict:
    """sp2_synchronize: wait for the handle's stream, complete the last call made
    with sync=False and return its info."""
    h = handle or default_handle()
    info = L.Info()
    h.check(h.lib.sp2_synchronize(h.h, C.byref(info)), allow_noconv)
    return info.to_dict()


def sp2_density(H, nocc: float, mode="bf16x2", out=None, handle: Handle | None = None,
                allow_noconv: bool = False, sync: bool = True, **kw):
    """D = theta(mu I - H) by SP2 (Eq. DM0). H: (N, N) float64/float32, torch
    CUDA tensor or numpy array. Returns (D, info dict); with sync=False (device
    buffers) the call returns without waiting and info is None."""
    h = handle or default_handle()
    h.bind_stream()
    n = H.shape[0]
    D = out if out is not None else _empty_like(H, (n, n))
    opts, _keep = make_opts(mode, **kw)
    info = _info_arg(sync)
    rc = h.lib.sp2_density(h.h, _ptr(H), n, _dtype_code(H), float(nocc), C.byref(opts), _ptr(D),
                           _info_ref(info))
    h.check(rc, allow_noconv)
    return D, _info_dict(info)


def sp2_response(H, nocc: float, H1, diag_only: bool = False, mode="bf16x2",
                 want_density: bool = False, handle: Handle | None = None,
                 allow_noconv: bool = False, sync: bool = True, **kw):
    """First-order responses D1_k to H1_k (Eq. DMPert). H1: (K, N, N), or
    (K, N) diagonals with diag_only=True. Returns (D1, D or None, info)."""
    h = handle or default_handle()
    h.bind_stream()
    n = H.shape[0]
    k = H1.shape[0]
    D1 = _empty_like(H, (k, n, n))
    D = _empty_like(H, (n, n)) if want_density else None
    opts, _keep = make_opts(mode, **kw)
    info = _info_arg(sync)
    rc = h.lib.sp2_response(h.h, _ptr(H), n, _dtype_code(H), float(nocc), _ptr(H1), k,
                            1 if diag_only else 0, C.byref(opts), _ptr(D), _ptr(D1),
                            _info_ref(info))
    h.check(rc, allow_noconv)
    return D1, D, _info_dict(info)


def sp2_susceptibility(H, nocc: float, A, direction: str = "forward", diag_only: bool = False,
                       mode="bf16x2", want_density: bool = False, handle: Handle | None = None,
                       allow_noconv: bool = False, out=None, D_out=None, sync: bool = True, **kw):
    """chi^A_l for observables A_l (L, N, N) or diagonals (L, N): forward
    Eq. DMSuscept, or backward Eq. DM2 with checkpointed X_n. Returns (chi, D or None, info).
    out / D_out: caller-owned result arrays (L, N, N) / (N, N) of H's dtype and kind,
    e.g. page-locked host memory for fast device-to-host copies."""
    h = handle or default_handle()
    h.bind_stream()
    n = H.shape[0]
    l = A.shape[0]
    chi = out if out is not None else _empty_like(H, (l, n, n))
    D = (D_out if D_out is not None else _empty_like(H, (n, n))) if want_density else None
    if tuple(chi.shape) != (l, n, n) or (D is not None and tuple(D.shape) != (n, n)):
        raise ValueError("out / D_out have the wrong shape")
    opts, _keep = make_opts(mode, **kw)
    info = _info_arg(sync)
    d = {"forward": 0, "backward": 1}[direction]
    rc = h.lib.sp2_susceptibility(h.h, _ptr(H), n, _dtype_code(H), float(nocc), _ptr(A), l,
                                  1 if diag_only else 0, d, C.byref(opts), _ptr(D), _ptr(chi),
                                  _info_ref(info))
    h.check(rc, allow_noconv)
    return chi, D, _info_dict(info)


def sp2_nonorth_susceptibility(H, S, nocc: float, A, mode="fp64", want_z: bool = False,
                               handle: Handle | None = None, **kw):
    """Non-orthonormal basis (Sec. V.A): returns (D, W_H, W_S, Z or None, info)
    so that d Tr[A D] / d tau = Tr[A_t D] + Tr[W_H H_t] + Tr[W_S S_t] for any
    basis-set dependent perturbation (A_t, H_t, S_t)."""
    h = handle or default_handle()
    h.bind_stream()
    n = H.shape[0]
    D, WH, WS = (_empty_like(H, (n, n)) for _ in range(3))
    Z = _empty_like(H, (n, n)) if want_z else None
    opts, _keep = make_opts(mode, **kw)
    info = L.Info()
    rc = h.lib.sp2_nonorth_susceptibility(h.h, _ptr(H), _ptr(S), n, _dtype_code(H), float(nocc),
                                          _ptr(A), C.byref(opts), _ptr(D), _ptr(WH), _ptr(WS),
                                          _ptr(Z), C.byref(info))
    h.check(rc)
    return D, WH, WS, Z, info.to_dict()


def sp2_adjoint(G, handle: Handle, sync: bool = True):
    """Eq. DM2 for the symmetric part of G against the X_n history kept by the
    handle's last sp2_density(keep_history=True). Returns d Tr[G D]/dH."""
    h = handle
    h.bind_stream()
    n = G.shape[0]
    out = _empty_like(G, (n, n))
    info = _info_arg(sync)
    rc = h.lib.sp2_adjoint(h.h, _ptr(G), n, _dtype_code(G), _ptr(out), _info_ref(info))
    h.check(rc)
    return out


def sp2_fermi(H, mu: float, kT: float, B=None, diag_only: bool = False, canonical: bool = True,
              n_doublings: int = 20, mode="fp64", want_density: bool = True,
              handle: Handle | None = None, **kw):
    """Finite-temperature density f(H) and first-order responses to B_k
    (Sec. V.B; canonical: Tr[D1_k] = 0). B: (K, N, N) or (K, N) diagonals.
    Returns (D1 or None, D or None, info)."""
    h = handle or default_handle()
    h.bind_stream()
    n = H.shape[0]
    k = 0 if B is None else B.shape[0]
    D1 = _empty_like(H, (k, n, n)) if k else None
    D = _empty_like(H, (n, n)) if want_density else None
    opts, _keep = make_opts(mode, **kw)
    info = L.Info()
    rc = h.lib.sp2_fermi(h.h, _ptr(H), n, _dtype_code(H), float(mu), float(kT),
                         _ptr(B) if k else None, k, 1 if diag_only else 0, 1 if canonical else 0,
                         int(n_doublings), C.byref(opts), _ptr(D), _ptr(D1), C.byref(info))
    h.check(rc)
    return D1, D, info.to_dict()


def sp2_scf_response(H, nocc: float, norb: int, K, Vext, mixer: str = "linear",
                     alpha: float = 0.3, history: int = 8, tol: float = 1e-6, max_iter: int = 100,
                     W1=None, W2=None, bf16_infer: bool = True, record: bool = False,
                     mode="fp64", refine_mode=None, refine_below: float = 0.0,
                     kT: float = 0.0, mu: float = 0.0, n_doublings: int = 20,
                     canonical: bool = True,
                     handle: Handle | None = None, allow_noconv: bool = False,
                     return_info: bool = False, **kw):
    """Self-consistent site-charge response for F fields (rows of Vext, float64).
    K: (n_sites, n_sites) float64. Returns (q, residuals, iterations, (traj_r,
    traj_q) or None), plus the info dict when return_info; q and the
    trajectories live where Vext lives. refine_mode / refine_below: compute the
    responses in another arithmetic mode once the residual is below
    refine_below or stalls (info["refine_iter"] = first such iteration).
    kT > 0: finite-temperature responses at chemical potential mu (Sec. V.B;
    canonical mu_1 by default)."""
    h = handle or default_handle()
    h.bind_stream()
    n = H.shape[0]
    F, ns = Vext.shape
    so = L.ScfOpts()
    so.mixer = L.MIXERS[mixer]
    so.alpha = float(alpha)
    so.history = int(history)
    so.tol = float(tol)
    so.max_iter = int(max_iter)
    so.W1 = _ptr(W1) if W1 is not None else None
    so.W2 = _ptr(W2) if W2 is not None else None
    so.hidden = int(W1.shape[0]) if W1 is not None else 0
    so.bf16_infer = 1 if bf16_infer else 0
    so.kT = float(kT)
    so.mu = float(mu)
    so.n_doublings = int(n_doublings)
    so.canonical = 1 if canonical else 0
    if refine_mode is not None:
        so.refine_mode = L.MODES[refine_mode] if isinstance(refine_mode, str) else int(refine_mode)
        so.refine_below = float(refine_below)
    q = _empty_like(Vext, (F, ns))
    res = np.zeros(max_iter, dtype=np.float64)
    its = C.c_int(0)
    tr = tq = None
    if record:
        dev = Vext.device if isinstance(Vext, torch.Tensor) else "cuda"
        tr = torch.zeros((max_iter, F, ns), dtype=torch.float64, device=dev)
        tq = torch.zeros((max_iter, F, ns), dtype=torch.float64, device=dev)
    opts, _keep = make_opts(mode, **kw)
    info = L.Info()
    rc = h.lib.sp2_scf_response(h.h, _ptr(H), n, _dtype_code(H), float(nocc), int(norb), _ptr(K),
                                _ptr(Vext), F, C.byref(so), C.byref(opts), _ptr(q),
                                res.ctypes.data, C.byref(its), _ptr(tr) if record else None,
                                _ptr(tq) if record else None, C.byref(info))
    h.check(rc, allow_noconv)
    k = its.value
    out = (q, res[:k], k, ((tr[:k], tq[:k]) if record else None))
    return out + (info.to_dict(),) if return_info else out


def mlp_forward(W1, W2, X, bf16: bool = False, handle: Handle | None = None):
    """Y = relu(X W1^T) W2^T (device float32 tensors)."""
    h = handle or default_handle()
    h.bind_stream()
    Y = torch.empty((X.shape[0], W2.shape[0]), dtype=torch.float32, device=X.device)
    h.check(h.lib.sp2_mlp_forward(h.h, _ptr(W1), _ptr(W2), W1.shape[1], W1.shape[0], _ptr(X),
                                  X.shape[0], _ptr(Y), 1 if bf16 else 0))
    return Y


def mlp_loss_grad(W1, W2, X, T, handle: Handle | None = None):
    """(loss, dW1, dW2) of the mean squared error sum (Y - T)^2 / P."""
    h = handle or default_handle()
    h.bind_stream()
    g1 = torch.empty_like(W1)
    g2 = torch.empty_like(W2)
    loss = C.c_double(0.0)
    h.check(h.lib.sp2_mlp_loss_grad(h.h, _ptr(W1), _ptr(W2), W1.shape[1], W1.shape[0], _ptr(X),
                                    _ptr(T), X.shape[0], C.byref(loss), _ptr(g1), _ptr(g2)))
    return loss.value, g1, g2


def mlp_train(W1, W2, X, T, steps: int, lr: float, handle: Handle | None = None):
    """`steps` full-batch Adam steps in place; returns the loss history."""
    h = handle or default_handle()
    h.bind_stream()
    hist = np.zeros(max(steps, 1), dtype=np.float64)
    h.check(h.lib.sp2_mlp_train(h.h, _ptr(W1), _ptr(W2), W1.shape[1], W1.shape[0], _ptr(X),
                                _ptr(T), X.shape[0], int(steps), float(lr), hist.ctypes.data))
    return hist[:steps]


def response_contract(P, Q, diag_only: bool = False, handle: Handle | None = None):
    """out[l, k] = sum_ij P_l[i,j] Q_k[i,j] in FP64 (Tr[chi_l H1_k] / Tr[A_l D1_k]).
    P: (L, N, N); Q: (K, N, N) or (K, N) diagonals. Returns an (L, K) float64
    array of the same kind (torch CUDA tensor or numpy) as P."""
    h = handle or default_handle()
    h.bind_stream()
    l, n = P.shape[0], P.shape[-1]
    k = Q.shape[0]
    if isinstance(P, torch.Tensor):
        out = torch.empty((l, k), dtype=torch.float64, device=P.device)
    else:
        out = np.empty((l, k), dtype=np.float64)
    if P.dtype != Q.dtype:
        raise TypeError("P and Q must have the same element type")
    rc = h.lib.response_contract(h.h, _ptr(P), l, _ptr(Q), k, n, _dtype_code(P),
                                 1 if diag_only else 0, _ptr(out))
    h.check(rc)
    return out
