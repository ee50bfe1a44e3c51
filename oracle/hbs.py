"""HBS compression, inverse build and inverse apply, plain numpy / scipy.

Test infrastructure only (see ``oracle/__init__``).

Paper:
* Tree (Sec. 3.2, Figs. 2-3): the root is the whole grid; level l -> l+1 cuts
  vertically when l is even (first child alpha = left, beta = right) and
  horizontally when l is odd (alpha = upper, i.e. larger x2, beta = lower);
  2^L equal leaves.  Node i of level l has children 2i, 2i+1 of level l+1.
* Compression (Sec. 3.2): row ID  G(I_tau, I_tau^c) ~ U_tau G(I_skel, I_tau^c)
  (Eq. (12)), computed from the proxy block G(I_tau, I_proxy) (Eq. (13)); the
  proxy set is the ring of lattice points at Chebyshev distance 1..w outside
  the box.  Parents use the children's skeletons as rows (Eq. (14)); sibling
  blocks are G_ab = G(skel_a, skel_b) (Eq. (15)).  The proxy block is the
  same for every box of a level (translation invariance), so one ID per level.
  V_tau = U_tau by symmetry of G; V* is read as the plain transpose U^T (G is
  complex symmetric, not Hermitian), so G_ba = G_ab^T.
* ID via CPQR (Sec. 2.1) of the transposed block; the local tolerance is
  eps * ||proxy block||_F (remark on the local tolerance, Sec. 3.2): the rank
  is the first k whose trailing R block has Frobenius norm <= that.
* Algorithm 1 (build): leaves X = (I + B G_leaf)^-1 (Eq. (20)),
  S = U^T X B U (Eq. (23)); parents X = [[I, S_a G_ab],[S_b G_ba, I]]^-1
  (Eq. (26)), S = U^T X diag(S_a, S_b) U (Eq. (27)); the root forms X only.
  The loop runs over every level l = L-1, ..., 0.
* Algorithm 2 (apply): up pass (Eqs. (24), (28)), root solve (Eq. (29)), down
  pass over l = 1, ..., L-1 with Lemma 4.1 (Eq. (18)), leaf recovery.
* The transposed apply (for the adjoint solve): the steps of Algorithm 2 in
  reverse order, each factor transposed.

Parity pins (tests/test_oracle_hbs.py): the ID property U(J,:) = I and its
accuracy on the full complement block; the Lemma 4.1 identity; the HBS inverse
against the dense inverse (error ~ eps, -> 0 as eps -> 0); Table 1's proxy
accuracy; the transposed apply by the bilinear identity y^T (M x) = (M^T y)^T x
and against the dense transpose of M assembled column by column; the Woodbury
local solution operator against the inverse of Eq. (26) (and the block as printed,
without the scattering matrices, against it: it fails).
"""
import numpy as np
import scipy.linalg as sla

from . import kernel, lattice


class Tree:
    """Uniform binary tree on an nx x ny grid with square leaves of side s."""

    def __init__(self, nx, ny, leaf):
        self.nx, self.ny, self.s = nx, ny, leaf
        L = 0
        w, h = nx, ny
        dims = [(w, h)]
        while (w, h) != (leaf, leaf):
            if L % 2 == 0:
                if w % 2:
                    raise ValueError("grid does not split into square leaves")
                w //= 2
            else:
                if h % 2:
                    raise ValueError("grid does not split into square leaves")
                h //= 2
            L += 1
            dims.append((w, h))
            if w < leaf or h < leaf:
                raise ValueError("grid does not split into square leaves")
        self.L = L
        self.dims = dims  # dims[l] = (width, height) of a level-l box
        self.offsets = []  # offsets[l] = (off_alpha, off_beta) for the cut l -> l+1
        for l in range(L):
            cw, ch = dims[l + 1]
            if l % 2 == 0:
                self.offsets.append((np.array([0, 0]), np.array([cw, 0])))
            else:
                self.offsets.append((np.array([0, ch]), np.array([0, 0])))
        self.origins = [np.zeros((1, 2), dtype=np.int64)]
        for l in range(L):
            oa, ob = self.offsets[l]
            par = self.origins[l]
            ch = np.empty((2 * len(par), 2), dtype=np.int64)
            ch[0::2] = par + oa
            ch[1::2] = par + ob
            self.origins.append(ch)


def box_points(w, h):
    """Local coordinates (lx, ly) of a w x h box, row-major (lx fastest)."""
    ly, lx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    return np.stack([lx.ravel(), ly.ravel()], axis=1)


def proxy_ring(w, h, width):
    """Lattice points at Chebyshev distance 1..width outside a w x h box."""
    ly, lx = np.meshgrid(np.arange(-width, h + width), np.arange(-width, w + width), indexing="ij")
    lx, ly = lx.ravel(), ly.ravel()
    outside = (lx < 0) | (lx >= w) | (ly < 0) | (ly >= h)
    return np.stack([lx[outside], ly[outside]], axis=1)


def kernel_block(kappa, h, order, P, Q):
    """Matrix entries G(p, q) = h^2 (G(h|q-p|) + tau_{q-p}) for local points
    P (rows) and Q (columns); tau only on the order-p stencil, h^2 tau_0 on
    coincident points (Eq. (10) with the corrections of Eq. (8))."""
    d = Q[None, :, :] - P[:, None, :]
    r = h * np.hypot(d[..., 0], d[..., 1])
    out = np.zeros(r.shape, dtype=np.complex128)
    nz = r > 0
    out[nz] = kernel.green(kappa, r[nz])
    pts, w = lattice.correction_weights(order, kappa * h)
    for (a, b), wt in zip(pts, w):
        out[(d[..., 0] == a) & (d[..., 1] == b)] += wt
    return h * h * out


def row_id(A, eps):
    """Row ID A ~ U A(J, :) by CPQR of A^T (Sec. 2.1).  Returns (J, U)."""
    m = A.shape[0]
    tol = eps * np.linalg.norm(A)
    _, R, perm = sla.qr(A.T, mode="economic", pivoting=True)
    r = R.shape[0]
    # trailing Frobenius norms of R[k:, k:] for k = 0..r
    tail = np.zeros(r + 1)
    for k in range(r - 1, -1, -1):
        tail[k] = np.sqrt(tail[k + 1] ** 2 + np.sum(np.abs(R[k, k:]) ** 2)
                          + np.sum(np.abs(R[k + 1:, k]) ** 2))
    k = next(i for i in range(r + 1) if tail[i] <= tol)
    T = sla.solve_triangular(R[:k, :k], R[:k, k:])
    U = np.zeros((m, k), dtype=np.complex128)
    U[perm[:k], np.arange(k)] = 1.0
    U[perm[k:], :] = T.T
    return perm[:k], U


def woodbury_local_solution(S_a, S_b, L_ab, R_ab, L_ba, R_ba):
    """Local solution operator of a parent by the Woodbury form of Sec. 4.1 (the
    remark after Algorithm 2, Eq. blockinv): with low-rank sibling blocks
    G_ab = L_ab R_ab^T and G_ba = L_ba R_ba^T (plain transposes: G is complex
    symmetric), X = [[I, S_a G_ab], [S_b G_ba, I]]^-1 (Eq. (26)) is
        X = I - P (I + Q P)^-1 Q,   P = diag(S_a L_ab, S_b L_ba),
                                     Q = [[0, R_ab^T], [R_ba^T, 0]],
    and the middle block I + Q P = [[I, R_ab^T S_b L_ba], [R_ba^T S_a L_ab, I]]
    carries the children's scattering matrices (the printed block omits them)."""
    k1, k2 = S_a.shape[0], S_b.shape[0]
    r1, r2 = L_ab.shape[1], L_ba.shape[1]
    P = np.zeros((k1 + k2, r1 + r2), dtype=complex)
    P[:k1, :r1] = S_a @ L_ab
    P[k1:, r1:] = S_b @ L_ba
    Q = np.zeros((r1 + r2, k1 + k2), dtype=complex)
    Q[:r1, k1:] = R_ab.T
    Q[r1:, :k1] = R_ba.T
    middle = np.eye(r1 + r2, dtype=complex) + Q @ P
    return np.eye(k1 + k2, dtype=complex) - P @ np.linalg.solve(middle, Q)


class Compression:
    """Per-level skeletons, U matrices and sibling blocks (one box per level)."""

    def __init__(self, kappa, h, tree, order, eps, ring):
        self.kappa, self.h, self.tree, self.order = kappa, h, tree, order
        L = tree.L
        self.skel = [None] * (L + 1)   # local coords within a level-l box
        self.U = [None] * (L + 1)      # rows_l x k_l
        self.rank = [0] * (L + 1)
        self.G_sib = [None] * (L + 1)  # G_sib[l] = G(skel_a, skel_b), children at level l
        for l in range(L, 0, -1):
            w, hh = tree.dims[l]
            if l == L:
                rows = box_points(w, hh)
            else:
                oa, ob = tree.offsets[l]
                rows = np.concatenate([self.skel[l + 1] + oa, self.skel[l + 1] + ob])
            A = kernel_block(kappa, h, order, rows, proxy_ring(w, hh, ring))
            J, U = row_id(A, eps)
            self.skel[l] = rows[J]
            self.U[l] = U
            self.rank[l] = len(J)
        for l in range(1, L + 1):
            oa, ob = tree.offsets[l - 1]
            self.G_sib[l] = kernel_block(kappa, h, order, self.skel[l] + oa, self.skel[l] + ob)
        s = tree.s
        self.G_leaf = kernel_block(kappa, h, order, box_points(s, s), box_points(s, s))


def gather_leaves(tree, x):
    """Grid vector(s) [..., ny*nx] -> leaf blocks [..., 2^L, s*s]."""
    s = tree.s
    xs = np.asarray(x).reshape(x.shape[:-1] + (tree.ny, tree.nx))
    pts = box_points(s, s)
    o = tree.origins[tree.L]
    iy = o[:, 1][:, None] + pts[None, :, 1]
    ix = o[:, 0][:, None] + pts[None, :, 0]
    return xs[..., iy, ix]


def scatter_leaves(tree, blocks):
    s = tree.s
    out = np.zeros(blocks.shape[:-2] + (tree.ny, tree.nx), dtype=blocks.dtype)
    pts = box_points(s, s)
    o = tree.origins[tree.L]
    iy = o[:, 1][:, None] + pts[None, :, 1]
    ix = o[:, 0][:, None] + pts[None, :, 0]
    out[..., iy, ix] = blocks
    return out.reshape(blocks.shape[:-2] + (tree.ny * tree.nx,))


class Inverse:
    """Algorithm 1 (build) and Algorithm 2 (apply) for I + B G."""

    def __init__(self, comp, b):
        t = comp.tree
        L = t.L
        kap2 = comp.kappa ** 2
        self.comp = comp
        self.Bleaf = kap2 * gather_leaves(t, np.asarray(b, dtype=np.float64).ravel())  # (2^L, s^2)
        self.X = [None] * (L + 1)
        self.S = [None] * (L + 1)
        # leaves: X = (I + B G)^-1, S = U^T X B U
        n = t.s * t.s
        Aleaf = np.eye(n)[None] + self.Bleaf[:, :, None] * comp.G_leaf[None]
        self.X[L] = np.linalg.inv(Aleaf)
        UL = comp.U[L]
        self.XBU = self.X[L] @ (self.Bleaf[:, :, None] * UL[None])
        self.S[L] = UL.T[None] @ self.XBU
        for l in range(L - 1, -1, -1):
            Sa, Sb = self.S[l + 1][0::2], self.S[l + 1][1::2]
            Gab = comp.G_sib[l + 1]
            k = Gab.shape[0]
            I = np.eye(k)[None].repeat(len(Sa), axis=0)
            K = np.block([[I, Sa @ Gab], [Sb @ Gab.T, I]])
            self.X[l] = np.linalg.inv(K)
            if l > 0:
                U = comp.U[l]
                DU = np.concatenate([Sa @ U[:k], Sb @ U[k:]], axis=1)
                self.S[l] = U.T[None] @ self.X[l] @ DU

    def apply(self, f):
        """q ~ (I + B G)^-1 f for f of shape [N] (Algorithm 2)."""
        comp, t = self.comp, self.comp.tree
        L = t.L
        fl = gather_leaves(t, np.asarray(f, dtype=np.complex128))[..., None]  # (2^L, n, 1)
        rt = [None] * (L + 1)
        r_leaf = self.X[L] @ fl
        rt[L] = comp.U[L].T[None] @ r_leaf
        for l in range(L - 1, 0, -1):  # upward pass
            rab = np.concatenate([rt[l + 1][0::2], rt[l + 1][1::2]], axis=1)
            rt[l] = comp.U[l].T[None] @ (self.X[l] @ rab)
        wt = [None] * (L + 1)
        # root: w = [[0, G_ab], [G_ba, 0]] X_root [r_a; r_b]
        q = self.X[0] @ np.concatenate([rt[1][0::2], rt[1][1::2]], axis=1)
        wt[1] = self._lemma(1, q, None)
        for l in range(1, L):  # downward pass
            k = self.comp.rank[l + 1]
            U = comp.U[l]
            Sa, Sb = self.S[l + 1][0::2], self.S[l + 1][1::2]
            Uw = U[None] @ wt[l]
            SUw = np.concatenate([Sa @ Uw[:, :k], Sb @ Uw[:, k:]], axis=1)
            rab = np.concatenate([rt[l + 1][0::2], rt[l + 1][1::2]], axis=1)
            q = self.X[l] @ (rab - SUw)
            wt[l + 1] = self._lemma(l + 1, q, Uw)
        ql = r_leaf - self.XBU @ wt[L]
        return scatter_leaves(t, ql[..., 0])

    def apply_transpose(self, g):
        """q = M^T g for the map M of ``apply`` (plain transpose, no conjugate).

        Algorithm 2 read backwards with every factor transposed (the adjoint of
        each step, in reverse order):
        * leaves: w~_L = -(X B U)^T g  (transpose of the leaf recovery);
        * upward through the downward pass, l = L-1, ..., 1: with Gamma the
          sibling map of Lemma 4.1 ([[0, G_ab], [G_ab^T, 0]], its own
          transpose), t_l = X_l^T Gamma w~_{l+1} (kept), then
          w~_l = U_l^T (w~_{l+1} - diag(S_a, S_b)^T t_l);
        * root: r~_1 = X_0^T Gamma w~_1;
        * downward through the upward pass, l = 1, ..., L-1:
          r~_{l+1} = t_l + X_l^T U_l r~_l;
        * leaves: q = X_L^T (g + U_L r~_L).
        """
        comp, t = self.comp, self.comp.tree
        L = t.L

        def T(a):
            return np.swapaxes(a, -1, -2)

        def pairs(x):  # children (2P, k, 1) -> parents (P, 2k, 1)
            return np.concatenate([x[0::2], x[1::2]], axis=1)

        def split(x):  # parents (P, 2k, 1) -> children (2P, k, 1)
            k = x.shape[1] // 2
            out = np.empty((2 * x.shape[0], k, x.shape[2]), dtype=x.dtype)
            out[0::2] = x[:, :k]
            out[1::2] = x[:, k:]
            return out

        gl = gather_leaves(t, np.asarray(g, dtype=np.complex128))[..., None]  # (2^L, n, 1)
        w = -(T(self.XBU) @ gl)
        tl = [None] * (L + 1)
        for l in range(L - 1, 0, -1):
            k = comp.rank[l + 1]
            qbar = pairs(self._lemma(l + 1, pairs(w), None))
            tl[l] = T(self.X[l]) @ qbar
            Sa, Sb = self.S[l + 1][0::2], self.S[l + 1][1::2]
            STt = np.concatenate([T(Sa) @ tl[l][:, :k], T(Sb) @ tl[l][:, k:]], axis=1)
            w = comp.U[l].T[None] @ (pairs(w) - STt)
        r = split(T(self.X[0]) @ pairs(self._lemma(1, pairs(w), None)))
        for l in range(1, L):
            r = split(tl[l] + T(self.X[l]) @ (comp.U[l][None] @ r))
        out = T(self.X[L]) @ (gl + comp.U[L][None] @ r)
        return scatter_leaves(t, out[..., 0])

    def _lemma(self, level, q, Uw):
        """Lemma 4.1: [w_a; w_b] = [[0, G_ab], [G_ba, 0]] [q_a; q_b] + U w_parent,
        returned interleaved as children (2i, 2i+1) of level `level`."""
        Gab = self.comp.G_sib[level]
        k = Gab.shape[0]
        wa = Gab[None] @ q[:, k:]
        wb = Gab.T[None] @ q[:, :k]
        if Uw is not None:
            wa = wa + Uw[:, :k]
            wb = wb + Uw[:, k:]
        out = np.empty((2 * q.shape[0], k, q.shape[2]), dtype=np.complex128)
        out[0::2] = wa
        out[1::2] = wb
        return out
