"""Learned factored preconditioner M^{-1} = G G^T for PCG.

The paper registers learned preconditioners as a future backend without a
design (Sec. 5).  This module drives the library's kernels (sla_mp_*,
sla_ggt_loss_grad, sla_adam_step, sla_cg_ggt): a message-passing network over
the matrix graph predicts G on the pattern of tril(A); PCG applies it as two
SpMVs; Jacobi-PCG is the fallback and the yardstick.  Every arithmetic step
runs in the CUDA library; this file only allocates buffers and sequences
calls.

Network (width 32; BF16 weights, FP32 accumulation, FP32 master weights):
  F = (sum_{j!=i}|e_ij|, sum_{j!=i} e_ij, deg_i/8),  e_ij = A_ij/sqrt(A_ii A_jj)
  H0 = relu(F W0^T + b0)
  3 x: Agg_i = sum_{j!=i} e_ij H_j;  H <- H + relu([H | Agg] W_l^T + c_l)
  [P | Q | R] = H Uh^T + bh
  G_ij = v.relu(P_i + Q_j + ue e_ij) / sqrt(A_ii)    (j < i, tril(A) pattern)
  G_ii = exp(vd.relu(R_i)) / sqrt(A_ii)
With v = vd = 0 (the initial state) G = D^{-1/2}: exactly Jacobi.

Training: systems generated by the library's own solver -- for each step a
system, b ~ N(0, I), x* from CG to rtol 1e-10 -- and the loss
(x* - G G^T b)^T A (x* - G G^T b) / (x*^T A x*).

Inference: the factor for a solve is the network's G with each column
divided by sqrt((G^T A G)_jj) (sla_ggt_normalize), the column scaling that
minimises Kaporin's condition number of G^T A G; it keeps the network's
off-diagonal pattern of weights and measured 9-27 % fewer iterations on the
unseen 2D systems.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np
import torch

from . import _lib as L
from . import sla

WIDTH = 32
LAYERS = 3
NFEAT = 3


def param_shapes() -> dict:
    s = {"W0": (WIDTH, NFEAT), "b0": (WIDTH,)}
    for l in range(LAYERS):
        s["W_%d" % l] = (WIDTH, 2 * WIDTH)
        s["c_%d" % l] = (WIDTH,)
    s.update({"Uh": (3 * WIDTH, WIDTH), "bh": (3 * WIDTH,), "ue": (WIDTH,), "v": (WIDTH,), "vd": (WIDTH,)})
    return s


def _bind():
    lib = L.lib()
    if getattr(lib, "_mp_bound", False):
        return lib
    P = ctypes.c_void_p
    i32, i64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    CSR = ctypes.POINTER(L.SlaCsr)
    CSRT = ctypes.POINTER(L.SlaCsrT)
    sz = ctypes.c_size_t
    sig = {
        "sla_mp_features": ([CSR, P, P, P, P, P], i32),
        "sla_tril_pattern": ([CSR, P, P, P, P, P, sz, P], i32),
        "sla_tril_pattern_ws": ([i32], sz),
        "sla_mp_dense_fwd": ([i32, i32, P, i32, P, i32, P, P, P, i32, P, P, P], i32),
        "sla_mp_dense_fwd_ex": ([i32, i32, P, i32, P, i32, P, P, P, i32, P, P, i32, P], i32),
        "sla_mp_tc_errors": ([P], i32),
        "sla_mp_dense_bwdx": ([i32, i32, P, i32, P, i32, i32, P, P, P], i32),
        "sla_mp_dense_bwdw": ([i32, i32, P, i32, P, i32, P, P, P, P, sz, P], i32),
        "sla_mp_dense_bwdw_ws": ([i32, i32], sz),
        "sla_mp_relu_mask": ([i64, P, P, P, P], i32),
        "sla_mp_aggregate": ([CSR, P, P, P, i32, P], i32),
        "sla_mp_head_fwd": ([i32, P, P, P, P, P, P, P, P, P, P, P, P], i32),
        "sla_mp_head_bwd": ([i32, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, sz, P], i32),
        "sla_mp_head_bwd_ws": ([i32], sz),
        "sla_ggt_loss_grad": ([CSR, P, CSR, P, CSRT, P, P, i32, P, P, P, sz, P], i32),
        "sla_ggt_loss_ws": ([i32], sz),
        "sla_ggt_normalize": ([CSR, P, CSR, CSRT, P, P, P], i32),
        "sla_ggt_normalize_bwd": ([CSR, P, CSR, CSRT, P, P, P, P], i32),
        "sla_fsai_factor": ([CSR, P, CSR, CSRT, P, P, P], i32),
        "sla_adam_step": ([i32, P, P, P, P, f32, f32, f32, f32, i32, f32, P, P], i32),
        "sla_to_bf16": ([i32, P, P, P], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    lib._mp_bound = True
    return lib


def _chk(name, rc):
    return L.check(name, rc)


def _p(t):
    return None if t is None else t.data_ptr()


class _Graph:
    """Per-system buffers: features, tril pattern G (+ its transpose), activations."""

    def __init__(self, A: sla.CSRMatrix, val: torch.Tensor):
        lib = _bind()
        dev = A.device
        n = A.n
        self.A, self.n, self.dev = A, n, dev
        st = sla._stream_ptr(dev)
        self.d = torch.empty(n, dtype=torch.float64, device=dev)
        self.e = torch.empty(max(A.nnz, 1), dtype=torch.float32, device=dev)
        self.F = torch.empty((n, NFEAT), dtype=torch.float32, device=dev)
        self.set_values(val)
        grp = torch.empty(n + 1, dtype=torch.int32, device=dev)
        gcol = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)
        gsrc = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)
        nnz_g = torch.empty(1, dtype=torch.int32, device=dev)
        ws = torch.empty(max(int(lib.sla_tril_pattern_ws(n)), 256), dtype=torch.uint8, device=dev)
        _chk("sla_tril_pattern", lib.sla_tril_pattern(ctypes.byref(A.c), grp.data_ptr(), gcol.data_ptr(),
                                                     gsrc.data_ptr(), nnz_g.data_ptr(), ws.data_ptr(),
                                                     ws.numel(), st))
        m = int(nnz_g.item())
        self.G = sla.CSRMatrix(grp, gcol[:m].clone(), check=False)
        self.gsrc = gsrc[:m].clone()
        sla.transpose_of(self.G)  # CSR of G^T: rowptr, row of each entry, entry index
        self.nnz_g = m
        f = lambda *shape: torch.empty(shape, dtype=torch.float32, device=dev)
        self.H = [f(n, WIDTH) for _ in range(LAYERS + 1)]
        self.H0pre = f(n, WIDTH)
        self.Agg = [f(n, WIDTH) for _ in range(LAYERS)]
        self.Z = [f(n, WIDTH) for _ in range(LAYERS)]
        self.PQR = f(n, 3 * WIDTH)
        self.theta = f(max(m, 1))
        self.g_val = torch.empty(max(m, 1), dtype=torch.float64, device=dev)
        # backward buffers
        self.dPQR = f(n, 3 * WIDTH)
        self.dtheta = f(max(m, 1))
        self.dH = [f(n, WIDTH) for _ in range(2)]
        self.dZ = f(n, WIDTH)
        self.dAgg = f(n, WIDTH)
        self.dG = torch.empty(max(m, 1), dtype=torch.float64, device=dev)
        self.g_norm = torch.empty(max(m, 1), dtype=torch.float64, device=dev)  # normalised factor (training)
        self.loss = torch.empty(2, dtype=torch.float64, device=dev)

    def set_values(self, val: torch.Tensor):
        """The value-dependent inputs (scaled entries and node features) for
        new values on the same pattern."""
        self.val = val
        _chk("sla_mp_features", _bind().sla_mp_features(ctypes.byref(self.A.c), val.data_ptr(), self.d.data_ptr(),
                                                       self.e.data_ptr(), self.F.data_ptr(),
                                                       sla._stream_ptr(self.dev)))


class LearnedPreconditioner:
    """The learned G G^T preconditioner: weights on one device and the
    forward / backward / training / solve entry points."""

    def __init__(self, device="cuda", seed: int = 0, params: dict | None = None):
        self.dev = torch.device(device)
        self.shapes = param_shapes()
        self.offsets = {}
        o = 0
        for k, shp in self.shapes.items():
            self.offsets[k] = (o, shp)
            o += int(np.prod(shp))
        self.np = o
        if params is None:
            rng = np.random.default_rng(seed)
            params = {}
            for k, shp in self.shapes.items():
                if len(shp) == 2:
                    params[k] = rng.standard_normal(shp) * np.sqrt(2.0 / shp[1]) * 0.5
                else:
                    params[k] = rng.standard_normal(shp) * 0.1
            params["v"][:] = 0.0
            params["vd"][:] = 0.0
        flat = np.concatenate([np.asarray(params[k], np.float64).ravel() for k in self.shapes])
        self.p = torch.tensor(flat, dtype=torch.float32, device=self.dev)
        self.pb = torch.empty(self.np, dtype=torch.bfloat16, device=self.dev)
        self.g = torch.zeros(self.np, dtype=torch.float32, device=self.dev)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.t = 0
        self._graphs = {}
        self._sync_bf16()
        self._ws = {}

    # -------------------------------------------------------------- params
    def _sync_bf16(self):
        _chk("sla_to_bf16", _bind().sla_to_bf16(self.np, self.p.data_ptr(), self.pb.data_ptr(),
                                                sla._stream_ptr(self.dev)))

    def view(self, name, which="p"):
        o, shp = self.offsets[name]
        buf = {"p": self.p, "pb": self.pb, "g": self.g}[which]
        return buf[o:o + int(np.prod(shp))].view(shp)

    def params_numpy(self, bf16: bool = False) -> dict:
        src = self.pb.float() if bf16 else self.p
        out = {}
        for k, (o, shp) in self.offsets.items():
            out[k] = src[o:o + int(np.prod(shp))].double().cpu().numpy().reshape(shp)
        return out

    def state_dict(self) -> dict:
        return {"params": self.p.detach().cpu().clone(), "t": self.t}

    def load_state_dict(self, sd: dict):
        self.p.copy_(sd["params"].to(self.dev))
        self.t = int(sd.get("t", 0))
        self._sync_bf16()

    def _scratch(self, key, nbytes):
        t = self._ws.get(key)
        if t is None or t.numel() < nbytes:
            t = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.dev)
            self._ws[key] = t
        return t

    # -------------------------------------------------------------- forward
    _GRAPH_CACHE = 4

    def graph(self, A: sla.CSRMatrix, val: torch.Tensor) -> _Graph:
        """Per-system buffers.  The pattern work (tril(A), the CSR of G^T) is
        kept for the last few matrices (by CSRMatrix object), so a factor for
        new values on a known pattern recomputes only the features."""
        key = id(A)
        hit = self._graphs.pop(key, None)
        if hit is not None and hit.A is A:
            hit.set_values(val)
            gr = hit
        else:
            gr = _Graph(A, val)
        self._graphs[key] = gr
        while len(self._graphs) > self._GRAPH_CACHE:
            self._graphs.pop(next(iter(self._graphs)))
        return gr

    def forward(self, gr: _Graph, inference: bool = False) -> torch.Tensor:
        """G values (FP64, on gr.G's pattern).  inference=True skips storing
        the pre-activations that only the backward pass reads."""
        lib = _bind()
        st = sla._stream_ptr(self.dev)
        n = gr.n
        pb = lambda k: self.view(k, "pb").data_ptr()
        pf = lambda k: self.view(k, "p").data_ptr()
        pre = (lambda t: None) if inference else (lambda t: t.data_ptr())
        _chk("dense0", lib.sla_mp_dense_fwd(n, NFEAT, gr.F.data_ptr(), 0, None, WIDTH, pb("W0"), pf("b0"), None, 1,
                                            pre(gr.H0pre), gr.H[0].data_ptr(), st))
        for l in range(LAYERS):
            _chk("agg", lib.sla_mp_aggregate(ctypes.byref(gr.A.c), gr.e.data_ptr(), gr.H[l].data_ptr(),
                                             gr.Agg[l].data_ptr(), 0, st))
            _chk("dense", lib.sla_mp_dense_fwd(n, WIDTH, gr.H[l].data_ptr(), WIDTH, gr.Agg[l].data_ptr(), WIDTH,
                                               pb("W_%d" % l), pf("c_%d" % l), gr.H[l].data_ptr(), 1,
                                               pre(gr.Z[l]), gr.H[l + 1].data_ptr(), st))
        _chk("head_dense", lib.sla_mp_dense_fwd(n, WIDTH, gr.H[LAYERS].data_ptr(), 0, None, 3 * WIDTH, pb("Uh"),
                                                pf("bh"), None, 0, None, gr.PQR.data_ptr(), st))
        _chk("head", lib.sla_mp_head_fwd(n, gr.G.rowptr.data_ptr(), gr.G.col.data_ptr(), gr.gsrc.data_ptr(),
                                         gr.e.data_ptr(), gr.d.data_ptr(), gr.PQR.data_ptr(), pf("ue"), pf("v"),
                                         pf("vd"), gr.theta.data_ptr(), gr.g_val.data_ptr(), st))
        return gr.g_val[:gr.nnz_g]

    # -------------------------------------------------------------- loss + backward
    def loss_grad(self, gr: _Graph, b: torch.Tensor, xstar: torch.Tensor, scale_free: bool = False,
                  g_val: torch.Tensor | None = None):
        """Loss (device FP64 scalar) and dloss/dG (gr.dG) of the factor with
        values g_val (default: the network's, gr.g_val).  scale_free: the
        A-norm error of the best multiple of G G^T b (sla_ggt_loss_grad
        mode 1), which PCG cannot tell from G G^T itself."""
        lib = _bind()
        ws = self._scratch("loss", lib.sla_ggt_loss_ws(gr.n))
        gv = gr.g_val if g_val is None else g_val
        _chk("sla_ggt_loss_grad", lib.sla_ggt_loss_grad(
            ctypes.byref(gr.A.c), gr.val.data_ptr(), ctypes.byref(gr.G.c), gv.data_ptr(),
            ctypes.byref(gr.G._transpose_c), b.data_ptr(), xstar.data_ptr(), 1 if scale_free else 0,
            gr.loss.data_ptr(), gr.dG.data_ptr(), ws.data_ptr(), ws.numel(), sla._stream_ptr(self.dev)))
        return gr.loss[0]

    def backward(self, gr: _Graph):
        """Gradient of the loss w.r.t. every parameter into self.g (FP32)."""
        lib = _bind()
        st = sla._stream_ptr(self.dev)
        n = gr.n
        pb = lambda k: self.view(k, "pb").data_ptr()
        pf = lambda k: self.view(k, "p").data_ptr()
        gf = lambda k: self.view(k, "g").data_ptr()
        wsh = self._scratch("head", lib.sla_mp_head_bwd_ws(n))
        hg = torch.empty(3 * WIDTH, dtype=torch.float32, device=self.dev)
        _chk("head_bwd", lib.sla_mp_head_bwd(
            n, gr.G.rowptr.data_ptr(), gr.G.col.data_ptr(), gr.gsrc.data_ptr(), gr.G._transpose[0].data_ptr(),
            gr.G._transpose[1].data_ptr(), gr.G._transpose[2].data_ptr(), gr.e.data_ptr(), gr.d.data_ptr(),
            gr.PQR.data_ptr(), pf("ue"), pf("v"), pf("vd"), gr.g_val.data_ptr(), gr.dG.data_ptr(),
            gr.dtheta.data_ptr(), gr.dPQR.data_ptr(), hg.data_ptr(), wsh.data_ptr(), wsh.numel(), st))
        self.view("v", "g").copy_(hg[0:WIDTH])
        self.view("ue", "g").copy_(hg[WIDTH:2 * WIDTH])
        self.view("vd", "g").copy_(hg[2 * WIDTH:])
        wsw = self._scratch("bwdw", lib.sla_mp_dense_bwdw_ws(3 * WIDTH, 2 * WIDTH))
        # head dense: [P|Q|R] = H3 Uh^T + bh
        dH, dHn = gr.dH[0], gr.dH[1]
        _chk("head_bwdx", lib.sla_mp_dense_bwdx(n, 3 * WIDTH, gr.dPQR.data_ptr(), WIDTH, pb("Uh"), 0, WIDTH, None,
                                                dH.data_ptr(), st))
        _chk("head_bwdw", lib.sla_mp_dense_bwdw(n, 3 * WIDTH, gr.dPQR.data_ptr(), WIDTH, gr.H[LAYERS].data_ptr(),
                                                0, None, gf("Uh"), gf("bh"), wsw.data_ptr(), wsw.numel(), st))
        for l in reversed(range(LAYERS)):
            # H_{l+1} = H_l + relu([H_l | Agg_l] W_l^T + c_l)
            _chk("mask", lib.sla_mp_relu_mask(n * WIDTH, dH.data_ptr(), gr.Z[l].data_ptr(), gr.dZ.data_ptr(), st))
            _chk("bwdx1", lib.sla_mp_dense_bwdx(n, WIDTH, gr.dZ.data_ptr(), WIDTH, pb("W_%d" % l), 0, 2 * WIDTH,
                                                dH.data_ptr(), dHn.data_ptr(), st))
            _chk("bwdx2", lib.sla_mp_dense_bwdx(n, WIDTH, gr.dZ.data_ptr(), WIDTH, pb("W_%d" % l), WIDTH, 2 * WIDTH,
                                                None, gr.dAgg.data_ptr(), st))
            _chk("bwdw", lib.sla_mp_dense_bwdw(n, WIDTH, gr.dZ.data_ptr(), WIDTH, gr.H[l].data_ptr(), WIDTH,
                                               gr.Agg[l].data_ptr(), gf("W_%d" % l), gf("c_%d" % l), wsw.data_ptr(),
                                               wsw.numel(), st))
            # Agg_l = E H_l with E symmetric: dH_l += E dAgg
            _chk("agg_bwd", lib.sla_mp_aggregate(ctypes.byref(gr.A.c), gr.e.data_ptr(), gr.dAgg.data_ptr(),
                                                 dHn.data_ptr(), 1, st))
            dH, dHn = dHn, dH
        # H0 = relu(F W0^T + b0)
        _chk("mask0", lib.sla_mp_relu_mask(n * WIDTH, dH.data_ptr(), gr.H0pre.data_ptr(), gr.dZ.data_ptr(), st))
        _chk("bwdw0", lib.sla_mp_dense_bwdw(n, WIDTH, gr.dZ.data_ptr(), NFEAT, gr.F.data_ptr(), 0, None, gf("W0"),
                                            gf("b0"), wsw.data_ptr(), wsw.numel(), st))
        return self.g

    def adam(self, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8, clip: float = 0.0):
        self.t += 1
        _chk("sla_adam_step", _bind().sla_adam_step(self.np, self.p.data_ptr(), self.g.data_ptr(),
                                                    self.m.data_ptr(), self.v.data_ptr(), lr, b1, b2, eps, self.t,
                                                    clip, self.pb.data_ptr(), sla._stream_ptr(self.dev)))

    # -------------------------------------------------------------- inference / solve
    def loss_grad_normalised(self, gr: _Graph, b: torch.Tensor, xstar: torch.Tensor, scale_free: bool = False):
        """The loss of the column-normalised factor (the one PCG uses) and
        its gradient w.r.t. the network's values in gr.dG: normalise into
        gr.g_norm, take the loss there, then sla_ggt_normalize_bwd."""
        lib = _bind()
        st = sla._stream_ptr(self.dev)
        _chk("sla_ggt_normalize", lib.sla_ggt_normalize(
            ctypes.byref(gr.A.c), gr.val.data_ptr(), ctypes.byref(gr.G.c), ctypes.byref(gr.G._transpose_c),
            gr.g_val.data_ptr(), gr.g_norm.data_ptr(), st))
        loss = self.loss_grad(gr, b, xstar, scale_free, g_val=gr.g_norm)
        _chk("sla_ggt_normalize_bwd", lib.sla_ggt_normalize_bwd(
            ctypes.byref(gr.A.c), gr.val.data_ptr(), ctypes.byref(gr.G.c), ctypes.byref(gr.G._transpose_c),
            gr.g_val.data_ptr(), gr.dG.data_ptr(), gr.dG.data_ptr(), st))
        return loss

    def normalize(self, gr: _Graph, g_val: torch.Tensor) -> torch.Tensor:
        """Columns of G divided by sqrt((G^T A G)_jj) (in place): the
        Kaporin-optimal column scaling, which the FSAI factor also has."""
        _chk("sla_ggt_normalize", _bind().sla_ggt_normalize(
            ctypes.byref(gr.A.c), gr.val.data_ptr(), ctypes.byref(gr.G.c), ctypes.byref(gr.G._transpose_c),
            g_val.data_ptr(), g_val.data_ptr(), sla._stream_ptr(self.dev)))
        return g_val

    def factor(self, A: sla.CSRMatrix, val: torch.Tensor, normalize: bool = True):
        """(G pattern as CSRMatrix, G values FP64) for a system: the network's
        G, with its columns normalised to diag(G^T A G) = I unless
        ``normalize`` is False."""
        gr = self.graph(A, val)
        gv = self.forward(gr, inference=True).clone()
        if normalize:
            self.normalize(gr, gv)
        return gr.G, gv

    def solve(self, A: sla.CSRMatrix, val: torch.Tensor, b: torch.Tensor, *, rtol: float = 1e-8,
              max_iter: int | None = None, factor=None, fallback: bool = True):
        """PCG with the learned G G^T.  If it does not converge (breakdown,
        not SPD, iteration cap) and ``fallback`` is set, Jacobi-PCG continues
        from the current iterate.  Returns (x, info, used_fallback)."""
        G, gv = self.factor(A, val) if factor is None else factor
        x, info = sla.cg_ggt(A, val, G, gv, b, rtol=rtol, max_iter=max_iter)
        if info.status != L.SLA_OK and fallback:
            x2, info2 = sla.cg(A, val, b, rtol=rtol, x0=x)
            return x2, info2, True
        return x, info, False


def tril_pattern(A: sla.CSRMatrix) -> sla.CSRMatrix:
    """The pattern of tril(A) as a CSRMatrix with its CSR of G^T (cached on A)."""
    G = getattr(A, "_tril_pattern", None)
    if G is None:
        lib = _bind()
        dev, n = A.device, A.n
        grp = torch.empty(n + 1, dtype=torch.int32, device=dev)
        gcol = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)
        gsrc = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)
        nnz_g = torch.empty(1, dtype=torch.int32, device=dev)
        ws = torch.empty(max(int(lib.sla_tril_pattern_ws(n)), 256), dtype=torch.uint8, device=dev)
        _chk("sla_tril_pattern", lib.sla_tril_pattern(ctypes.byref(A.c), grp.data_ptr(), gcol.data_ptr(),
                                                     gsrc.data_ptr(), nnz_g.data_ptr(), ws.data_ptr(),
                                                     ws.numel(), sla._stream_ptr(dev)))
        m = int(nnz_g.item())
        G = sla.CSRMatrix(grp, gcol[:m].clone(), check=False)
        sla.transpose_of(G)
        A._tril_pattern = G
    return G


def fsai_factor(A: sla.CSRMatrix, val: torch.Tensor):
    """The factored sparse approximate inverse on tril(A) (sla_fsai_factor):
    the classical factor of M^{-1} = G G^T the learned one is compared with.
    Returns (G pattern, G values FP64, columns that fell back to Jacobi)."""
    G = tril_pattern(A)
    gv = torch.empty(max(G.nnz, 1), dtype=torch.float64, device=A.device)
    fb = torch.zeros(1, dtype=torch.int32, device=A.device)
    _chk("sla_fsai_factor", _bind().sla_fsai_factor(ctypes.byref(A.c), val.data_ptr(), ctypes.byref(G.c),
                                                    ctypes.byref(G._transpose_c), gv.data_ptr(), fb.data_ptr(),
                                                    sla._stream_ptr(A.device)))
    return G, gv[:G.nnz], int(fb.item())


def training_system(k: int, n_lo: int = 64, n_hi: int = 128, seed0: int = 100000):
    """Training system k: 2D five-point diffusion on an N x N grid, N uniform
    in [n_lo, n_hi], faces exp(N(0, sigma^2)) with sigma ~ U[0.5, 2], all
    from seed seed0 + k."""
    from . import inputs as I
    rng = np.random.default_rng(seed0 + k)
    N = int(rng.integers(n_lo, n_hi + 1))
    sigma = float(rng.uniform(0.5, 2.0))
    return I.diffusion2d_random(N, seed0 + k, sigma)


def evaluate(model: LearnedPreconditioner, systems: int = 48, n_lo: int = 64, n_hi: int = 128,
             seed0: int = 100000, rhs: int = 2, normalize: bool = True, scale_free: bool = True,
             fsai: bool = False) -> float:
    """Mean training loss of the factor over the training systems (rhs fresh
    b ~ N(0, I) each, x* by the library's CG at rtol 1e-10): by default the
    scale-free loss of the column-normalised factor, i.e. of the
    preconditioner as PCG uses it.  fsai=True evaluates the classical FSAI
    factor (already normalised) on the same pattern instead."""
    dev = model.dev
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed0 + 7)
    acc = []
    for k in range(systems):
        rp, c, v = training_system(k, n_lo, n_hi, seed0)
        A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
        vt = torch.from_numpy(v).to(dev)
        gr = model.graph(A, vt)
        if fsai:
            gr.g_val[:gr.nnz_g].copy_(fsai_factor(A, vt)[1])
        else:
            model.forward(gr, inference=True)
            if normalize:
                model.normalize(gr, gr.g_val[:gr.nnz_g])
        for _ in range(rhs):
            b = torch.randn(A.n, dtype=torch.float64, device=dev, generator=gen)
            xs, _ = sla.cg(A, vt, b, rtol=1e-10)
            acc.append(model.loss_grad(gr, b, xs, scale_free).clone())
    return float(torch.stack(acc).mean())


def train(model: LearnedPreconditioner, systems: int = 64, steps: int = 400, lr: float = 3e-3,
          n_lo: int = 64, n_hi: int = 128, seed0: int = 100000, log_every: int = 50, clip: float = 1.0,
          verbose: bool = False, scale_free: bool = False, normalised: bool = False):
    """Trains on `systems` generated systems for `steps` steps; every step
    draws one system and a fresh b ~ N(0, I), solves it with the library's
    CG (rtol 1e-10) for x*, and takes one Adam step on the loss (the
    scale-free loss with scale_free=True; of the column-normalised factor,
    through the normalisation's backward, with normalised=True).  Returns
    the loss history (host floats, every `log_every` steps averaged)."""
    dev = model.dev
    pool = []
    for k in range(systems):
        rp, c, v = training_system(k, n_lo, n_hi, seed0)
        A = sla.CSRMatrix.from_numpy(rp, c, device=dev)
        vt = torch.from_numpy(v).to(dev)
        pool.append((A, vt, model.graph(A, vt)))
    rng = np.random.default_rng(seed0 - 1)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed0)
    hist, acc = [], []
    t0 = time.time()
    for s in range(steps):
        A, vt, gr = pool[int(rng.integers(len(pool)))]
        b = torch.randn(A.n, dtype=torch.float64, device=dev, generator=gen)
        xs, info = sla.cg(A, vt, b, rtol=1e-10)
        model.forward(gr)
        if normalised:
            loss = model.loss_grad_normalised(gr, b, xs, scale_free)
        else:
            loss = model.loss_grad(gr, b, xs, scale_free)
        model.backward(gr)
        model.adam(lr=lr, clip=clip)
        acc.append(loss)
        if (s + 1) % log_every == 0:
            hist.append(float(torch.stack(acc).mean()))
            acc = []
            if verbose:
                print("step %d loss %.4f (%.1fs)" % (s + 1, hist[-1], time.time() - t0), flush=True)
    return hist
