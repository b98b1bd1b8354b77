"""FP64 CPU oracle of the learned factored preconditioner (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s reference leg
may import this module; it shares no code with the CUDA library.

The paper names learned preconditioners as future work and gives no design
(Sec. 5); this module writes out, with plain PyTorch CPU ops in float64 and
autograd for the gradients, the design the CUDA kernels implement:

* Scaled system: d_i = A_ii, e_k = A_ij / sqrt(d_i d_j) for every stored
  entry k = (i, j).
* Node features (3): sum_{j != i} |e_ij|, sum_{j != i} e_ij, deg_i / 8.
* Input layer: H = relu(F W0^T + b0), width 32.
* Three message-passing layers, W_l = [W1 | W2] (32 x 64):
      Agg_i = sum_{j != i} e_ij H_j,   H <- H + relu([H | Agg] W_l^T + c_l).
* Head on the pattern of tril(A), [P | Q | R] = H Uh^T + bh (Uh 96 x 32):
      off-diagonal (i, j), j < i: theta = v . relu(P_i + Q_j + ue e_ij)
      diagonal: theta_ii = vd . relu(R_i)
      Gt_ii = exp(theta_ii), Gt_ij = theta_ij,  G = D^{-1/2} Gt  (row scaling),
  so that G G^T = D^{-1/2} Gt Gt^T D^{-1/2}; with v = vd = 0, G = D^{-1/2} and
  G G^T is the Jacobi preconditioner exactly.
* Training loss for one system and right-hand side b with x* = A^{-1} b and
  y = G G^T b:
      loss = (x* - k y)^T A (x* - k y) / (x*^T A x*),
  with k = 1, or in the scale-free form k = x*^T A y / y^T A y, the k that
  minimises it (the error of the best multiple of G G^T; PCG's iterates do
  not change when the preconditioner is scaled).  Its gradient here is
  autograd's through k as well.
* Column normalisation of the factor the network proposes (applied when the
  factor is formed for a solve): column j of G is divided by
  sqrt((G^T A G)_jj) = sqrt(sum_{i,k} G_ij A_ik G_kj), so that diag(G^T A G)
  = I.  Over all positive column scalings this minimises Kaporin's condition
  number (tr(G^T A G)/n)^n / det(G^T A G) of the preconditioned operator
  (arithmetic-geometric mean inequality; det is scaled by the product of the
  squared scales, tr is minimised relative to it at equal diagonals), the
  normalisation that the factored sparse approximate inverse (FSAI) built
  column by column also satisfies.
"""
from __future__ import annotations

import numpy as np
import torch

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


def init_params(seed: int = 0, zero_head: bool = True) -> dict:
    """Scaled-normal initial weights (numpy float64); the output vectors v and
    vd start at zero so that the initial G is the Jacobi factor."""
    rng = np.random.default_rng(seed)
    out = {}
    for k, shp in param_shapes().items():
        if len(shp) == 2:
            out[k] = rng.standard_normal(shp) * np.sqrt(2.0 / shp[1]) * 0.5
        else:
            out[k] = rng.standard_normal(shp) * 0.1
    if zero_head:
        out["v"][:] = 0.0
        out["vd"][:] = 0.0
    return out


def tril_pattern(rp, c):
    """CSR of the lower triangle (diagonal included) and, for each of its
    entries, the index of the same entry in A."""
    n = len(rp) - 1
    rows, cols, src = [], [], []
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            if c[k] <= i:
                rows.append(i)
                cols.append(c[k])
                src.append(k)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, np.asarray(rows, np.int64) + 1, 1)
    return np.cumsum(rowptr).astype(np.int32), np.asarray(cols, np.int32), np.asarray(src, np.int64)


def _graph(rp, c, v):
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    d = np.zeros(n)
    np.add.at(d, rows[rows == c], v[rows == c])
    e = v / np.sqrt(d[rows] * d[c])
    return n, rows, torch.tensor(d), torch.tensor(e)


def forward(params: dict, rp, c, v):
    """G on the tril(A) pattern: returns (g_rowptr, g_col, g_val float64 tensor)."""
    P = {k: (t if isinstance(t, torch.Tensor) else torch.tensor(t)) for k, t in params.items()}
    n, rows, d, e = _graph(rp, c, v)
    rows_t = torch.tensor(rows)
    cols_t = torch.tensor(np.asarray(c, np.int64))
    off = rows_t != cols_t
    # node features
    F = torch.zeros((n, NFEAT), dtype=torch.float64)
    F[:, 0] = torch.zeros(n, dtype=torch.float64).index_add(0, rows_t[off], e[off].abs())
    F[:, 1] = torch.zeros(n, dtype=torch.float64).index_add(0, rows_t[off], e[off])
    F[:, 2] = torch.zeros(n, dtype=torch.float64).index_add(0, rows_t[off], torch.ones(int(off.sum()), dtype=torch.float64)) / 8.0
    H = torch.relu(F @ P["W0"].T + P["b0"])
    for l in range(LAYERS):
        msg = e[off][:, None] * H[cols_t[off]]
        agg = torch.zeros_like(H).index_add(0, rows_t[off], msg)
        H = H + torch.relu(torch.cat([H, agg], dim=1) @ P["W_%d" % l].T + P["c_%d" % l])
    grp, gcol, src = tril_pattern(rp, c)
    src_t = torch.tensor(src)
    gi = rows_t[src_t]
    gj = cols_t[src_t]
    diag = gi == gj
    PQR = H @ P["Uh"].T + P["bh"]
    Pn, Qn, Rn = PQR[:, :WIDTH], PQR[:, WIDTH:2 * WIDTH], PQR[:, 2 * WIDTH:]
    hid = torch.relu(Pn[gi] + Qn[gj] + e[src_t][:, None] * P["ue"])
    theta_off = hid @ P["v"]
    hid_d = torch.relu(Rn[gi])
    theta_d = hid_d @ P["vd"]
    gt = torch.where(diag, torch.exp(theta_d), theta_off)
    g_val = gt / torch.sqrt(d[gi])
    return grp, gcol, g_val


def column_normalize(grp, gcol, g_val, rp, c, v):
    """Columns of G (CSR grp, gcol, g_val) divided by sqrt((G^T A G)_jj),
    written out with plain loops: for every column j, the entries G_ij of
    that column and the stored A_ik between their rows.  A column whose
    quadratic form is not positive and finite is left as it is."""
    n = len(grp) - 1
    g = np.asarray(g_val, dtype=np.float64)
    A = {}
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[(i, int(c[k]))] = A.get((i, int(c[k])), 0.0) + float(v[k])
    cols = {}
    for i in range(n):
        for e in range(grp[i], grp[i + 1]):
            cols.setdefault(int(gcol[e]), []).append((i, e))
    out = g.copy()
    for j, ent in cols.items():
        q = 0.0
        for (i, ei) in ent:
            for (k, ek) in ent:
                q += g[ei] * A.get((i, k), 0.0) * g[ek]
        if q > 0.0 and np.isfinite(q):
            for (_, e) in ent:
                out[e] = g[e] / np.sqrt(q)
    return out


def column_normalize_t(grp, gcol, g_val, rp, c, v):
    """The same normalisation with torch operations (differentiable in the
    float64 tensor g_val), through dense matrices: Gn = G diag(q)^{-1/2},
    q = diag(G^T A G), columns with q not positive and finite left as they
    are; returns Gn's values in g_val's order.  For small systems (tests)."""
    n = len(grp) - 1
    rows = torch.tensor(np.repeat(np.arange(n), np.diff(grp)))
    cols = torch.tensor(np.asarray(gcol, np.int64))
    G = torch.zeros((n, n), dtype=torch.float64).index_put((rows, cols), g_val, accumulate=True)
    Ad = torch.zeros((n, n), dtype=torch.float64)
    ar = torch.tensor(np.repeat(np.arange(n), np.diff(rp)))
    Ad = Ad.index_put((ar, torch.tensor(np.asarray(c, np.int64))), torch.tensor(np.asarray(v, np.float64)),
                      accumulate=True)
    q = torch.einsum("ij,ik,kj->j", G, Ad, G)
    ok = (q > 0.0) & torch.isfinite(q)
    scale = torch.where(ok, 1.0 / torch.sqrt(torch.where(ok, q, torch.ones_like(q))), torch.ones_like(q))
    return g_val * scale[cols]


def fsai_factor(rp, c, v):
    """The factored sparse approximate inverse on the pattern of tril(A)
    (Kolotilina and Yeremin), the classical non-learned G of M^{-1} = G G^T
    that the learned factor is compared with: column i of G solves
    A[P, P] y = e_1 on P = {j >= i : A_ji != 0} (ascending, i first) and is
    y / sqrt(y_1), so that (G^T A G)_ii = 1.  Dense numpy per column.
    Returns G as a dense [n, n] array."""
    n = len(rp) - 1
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[i, c[k]] += v[k]
    G = np.zeros((n, n))
    for i in range(n):
        P = [j for j in range(i, n) if A[j, i] != 0.0]
        y = np.linalg.solve(A[np.ix_(P, P)], np.eye(len(P))[0])
        G[P, i] = y / np.sqrt(y[0])
    return G


def ggt_apply(grp, gcol, g_val, u):
    """y = G (G^T u) with G given on a CSR pattern (differentiable in g_val, u)."""
    n = len(grp) - 1
    rows = torch.tensor(np.repeat(np.arange(n), np.diff(grp)))
    cols = torch.tensor(np.asarray(gcol, np.int64))
    s = torch.zeros(n, dtype=torch.float64).index_add(0, cols, g_val * u[rows])   # G^T u
    return torch.zeros(n, dtype=torch.float64).index_add(0, rows, g_val * s[cols])  # G s


def loss(grp, gcol, g_val, rp, c, v, b, xstar, scale_free=False):
    """(x* - k y)^T A (x* - k y) / (x*^T A x*), y = G G^T b; k = 1, or with
    scale_free the minimising k = x*^T A y / y^T A y (0 when y = 0)."""
    n = len(rp) - 1
    rows = torch.tensor(np.repeat(np.arange(n), np.diff(rp)))
    cols = torch.tensor(np.asarray(c, np.int64))
    vt = torch.tensor(v)
    bt = torch.as_tensor(b, dtype=torch.float64)
    xs = torch.as_tensor(xstar, dtype=torch.float64)

    def amul(z):
        return torch.zeros(n, dtype=torch.float64).index_add(0, rows, vt * z[cols])

    y = ggt_apply(grp, gcol, g_val, bt)
    if scale_free:
        Ay = amul(y)
        yAy = y @ Ay
        k = (xs @ Ay) / yAy if float(yAy.detach()) > 0.0 else torch.zeros((), dtype=torch.float64)
        y = k * y
    err = xs - y
    return (err @ amul(err)) / (xs @ bt)


def loss_and_grads(params: dict, rp, c, v, b, xstar, scale_free=False):
    """Loss and its gradient w.r.t. every parameter (autograd, float64)."""
    P = {k: torch.tensor(np.asarray(t, np.float64), requires_grad=True) for k, t in params.items()}
    grp, gcol, gv = forward(P, rp, c, v)
    L = loss(grp, gcol, gv, rp, c, v, b, xstar, scale_free)
    L.backward()
    return float(L.detach()), {k: t.grad.numpy().copy() for k, t in P.items()}, gv.detach().numpy()
