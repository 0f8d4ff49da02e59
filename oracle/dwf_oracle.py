"""FP64 CPU oracle for the even-odd preconditioned domain-wall Dirac operator, plain CG on
the normal equations and the multisplitting preconditioned CG (MSPCG).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  It shares no code with the CUDA path.

Every operator is written over the whole lattice with ``numpy.roll`` shifts and small dense
matrices, in complex128.  Field shapes (lexicographic, x fastest):

* 4D fermion ``(T, Z, Y, X, 4, 3)``; 5D fermion ``(Ls, T, Z, Y, X, 4, 3)``;
* links ``(T, Z, Y, X, 4, 3, 3)`` with mu = 0..3 = x, y, z, t;
* even-half vectors ``(Ls, V/2, 4, 3)``: the even sites (x+y+z+t even) in lexicographic order.

What the paper fixes and what is a reading (the paper does not print the operator):

* The paper's problem: DWF is Wilson times a fifth dimension and is not Hermitian, so CG
  runs on the normal equations A = D^dag D (Sec. 2.2, Eq. 3).  The operator itself is the
  standard Moebius domain-wall operator (reading):
    D_W(-M5) = (4 - M5) - Dh/2,
    Dh psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu),
    (K psi)_s = P- psi_{s+1} + P+ psi_{s-1},  psi_{Ls} = -mf psi_0,  psi_{-1} = -mf psi_{Ls-1},
    D+ = b + c K,  D- = 1 - K,  D = D_W D+ + D-   (Shamir: b = 1, c = 0).
* Chiral gamma basis: gamma_k = [[0, -i s_k], [i s_k, 0]], gamma_4 = [[0, 1], [1, 0]],
  gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1), P+- = (1 +- gamma_5)/2.
  Periodic boundary conditions in all four directions.
* Even-odd Schur complement on even sites (reading):
    M5op = (4 - M5) D+ + D-,
    Mpc = M5op - 1/4 Dh_eo D+ M5op^-1 Dh_oe D+,   A = Mpc^dag Mpc, solved as A x = phi.
* MSPCG (Sec. 2.3, Eqs. 4-5): preconditioned CG whose preconditioner is M = direct sum of the
  block-diagonal pieces A_s, applied as l plain CG iterations per block from a zero guess.
  Two readings of A_s: local_op="exact" is P_s A P_s, the diagonal block of A itself (Eq. 5:
  M keeps the diagonal blocks of A and has zero off-diagonal blocks); local_op="drop" is
  Mpc^dag Mpc built with every link whose two ends lie in different blocks set to zero
  (hopping across block faces dropped).  beta is Fletcher-Reeves unless flexible=True (Polak-Ribiere).

Every function here is pinned by a test in tests/test_oracle.py (no function is unpinned).
* Cost arithmetic of Sec. 4.1, Eqs. 6-7.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# ----------------------------------------------------------------------------------------
# Gamma matrices (chiral basis) and chiral projectors.
# ----------------------------------------------------------------------------------------
_S = [np.array([[0, 1], [1, 0]], dtype=complex),
      np.array([[0, -1j], [1j, 0]], dtype=complex),
      np.array([[1, 0], [0, -1]], dtype=complex)]
_Z2 = np.zeros((2, 2), dtype=complex)
_I2 = np.eye(2, dtype=complex)

GAMMA = np.array([np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in _S]
                 + [np.block([[_Z2, _I2], [_I2, _Z2]])])          # gamma_1..gamma_4 (x,y,z,t)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=complex)
P_PLUS = (ID4 + GAMMA5) / 2
P_MINUS = (ID4 - GAMMA5) / 2


@dataclass(frozen=True)
class DWFParams:
    dims: tuple          # (X, Y, Z, T)
    Ls: int
    M5: float
    mf: float
    b: float = 1.0
    c: float = 0.0


# ----------------------------------------------------------------------------------------
# Lattice helpers.
# ----------------------------------------------------------------------------------------
def _site_axis(field: np.ndarray, mu: int, trailing: int) -> int:
    """Array axis of direction mu for a field whose last `trailing` axes are internal."""
    # Lattice axes are (..., T, Z, Y, X, internal...): X is the last lattice axis.
    return field.ndim - trailing - 1 - mu


def shift(field: np.ndarray, mu: int, step: int, trailing: int) -> np.ndarray:
    """Returns f(x + step * mu_hat) (periodic)."""
    return np.roll(field, -step, axis=_site_axis(field, mu, trailing))


def parity(dims) -> np.ndarray:
    """(x+y+z+t) mod 2 on the (T, Z, Y, X) grid."""
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X),
                             indexing="ij")
    return (x + y + z + t) % 2


def spin_mul(m: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Applies a 4x4 spin matrix to a fermion field (spin axis is -2)."""
    return np.einsum("ab,...bc->...ac", m, psi)


def color_mul(u: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Applies the per-site 3x3 colour matrix u (T,Z,Y,X,3,3) to psi (...,T,Z,Y,X,4,3)."""
    return np.einsum("tzyxab,...tzyxsb->...tzyxsa", u, psi)


def dagger(u: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(u, -1, -2))


# ----------------------------------------------------------------------------------------
# Wilson hopping term and the Wilson operator (Sec. 2.2: DWF = Wilson x fifth dimension).
# ----------------------------------------------------------------------------------------
def hop(U: np.ndarray, psi: np.ndarray, dag: bool = False) -> np.ndarray:
    """Dh psi = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu).

    dag=True gives Dh^dag, the same sum with the two projector signs exchanged.
    psi may be 4D or 5D (any leading axes before T).
    """
    out = np.zeros_like(psi)
    sgn = 1.0 if dag else -1.0
    for mu in range(4):
        u_mu = U[..., mu, :, :]                                    # (T,Z,Y,X,3,3)
        fwd = color_mul(u_mu, shift(psi, mu, +1, 2))               # U_mu(x) psi(x+mu)
        u_back = np.roll(u_mu, 1, axis=3 - mu)                     # U_mu(x-mu)
        bwd = color_mul(dagger(u_back), shift(psi, mu, -1, 2))     # U_mu(x-mu)^dag psi(x-mu)
        out += spin_mul(ID4 + sgn * GAMMA[mu], fwd) + spin_mul(ID4 - sgn * GAMMA[mu], bwd)
    return out


def wilson(U: np.ndarray, psi: np.ndarray, M5: float, dag: bool = False) -> np.ndarray:
    """D_W(-M5) psi = (4 - M5) psi - Dh psi / 2."""
    return (4.0 - M5) * psi - 0.5 * hop(U, psi, dag)


# ----------------------------------------------------------------------------------------
# Fifth dimension: K, D+, D-, M5op as per-chirality real Ls x Ls matrices.
# ----------------------------------------------------------------------------------------
def shift_matrices(Ls: int, mf: float):
    """S_up psi_s = psi_{s+1} (psi_Ls = -mf psi_0); S_dn psi_s = psi_{s-1} (psi_-1 = -mf psi_Ls-1)."""
    up = np.zeros((Ls, Ls))
    dn = np.zeros((Ls, Ls))
    for s in range(Ls):
        if s + 1 < Ls:
            up[s, s + 1] = 1.0
        else:
            up[s, 0] = -mf
        if s - 1 >= 0:
            dn[s, s - 1] = 1.0
        else:
            dn[s, Ls - 1] = -mf
    return up, dn


def k_matrices(Ls: int, mf: float) -> np.ndarray:
    """K per chirality: [0] acts on the P+ components (spins 0,1), [1] on P- (spins 2,3).

    (K psi)_s = P- psi_{s+1} + P+ psi_{s-1}: on P+ rows K = S_dn, on P- rows K = S_up.
    """
    up, dn = shift_matrices(Ls, mf)
    return np.array([dn, up])


def s_apply(mats: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Applies per-chirality Ls x Ls matrices mats[chi] along the s axis (axis 0) of psi."""
    out = np.empty_like(psi)
    out[..., 0:2, :] = np.einsum("st,t...->s...", mats[0], psi[..., 0:2, :])
    out[..., 2:4, :] = np.einsum("st,t...->s...", mats[1], psi[..., 2:4, :])
    return out


def dplus_matrices(p: DWFParams) -> np.ndarray:
    return p.b * np.eye(p.Ls)[None] + p.c * k_matrices(p.Ls, p.mf)


def dminus_matrices(p: DWFParams) -> np.ndarray:
    return np.eye(p.Ls)[None] - k_matrices(p.Ls, p.mf)


def m5op_matrices(p: DWFParams) -> np.ndarray:
    """M5op = (4 - M5) D+ + D-, the even-even (= odd-odd) block of D."""
    return (4.0 - p.M5) * dplus_matrices(p) + dminus_matrices(p)


def m5op_inv_matrices(p: DWFParams) -> np.ndarray:
    m = m5op_matrices(p)
    return np.array([np.linalg.inv(m[0]), np.linalg.inv(m[1])])


def transpose_chi(mats: np.ndarray) -> np.ndarray:
    """Adjoint of a real per-chirality s-matrix (the matrices are real, chirality is kept)."""
    return np.swapaxes(mats, -1, -2)


# ----------------------------------------------------------------------------------------
# The full 5D domain-wall operator.
# ----------------------------------------------------------------------------------------
def dwf(U: np.ndarray, psi: np.ndarray, p: DWFParams, dag: bool = False) -> np.ndarray:
    """D = D_W(-M5) D+ + D-  (dag: D^dag = D+^dag D_W^dag + D-^dag).  psi: (Ls,T,Z,Y,X,4,3)."""
    dp, dm = dplus_matrices(p), dminus_matrices(p)
    if not dag:
        return wilson(U, s_apply(dp, psi), p.M5) + s_apply(dm, psi)
    return s_apply(transpose_chi(dp), wilson(U, psi, p.M5, dag=True)) + \
        s_apply(transpose_chi(dm), psi)


# ----------------------------------------------------------------------------------------
# Even-half packing.
# ----------------------------------------------------------------------------------------
def to_half(psi: np.ndarray, dims, par: int = 0) -> np.ndarray:
    """(Ls,T,Z,Y,X,4,3) -> (Ls, V/2, 4, 3): the sites of parity `par` in lexicographic order."""
    Ls = psi.shape[0]
    flat = psi.reshape(Ls, -1, 4, 3)
    sel = parity(dims).reshape(-1) == par
    return flat[:, sel].copy()


def from_half(h: np.ndarray, dims, par: int = 0) -> np.ndarray:
    """(Ls, V/2, 4, 3) -> (Ls,T,Z,Y,X,4,3), zero on the other parity."""
    X, Y, Z, T = dims
    Ls = h.shape[0]
    flat = np.zeros((Ls, X * Y * Z * T, 4, 3), dtype=complex)
    sel = parity(dims).reshape(-1) == par
    flat[:, sel] = h
    return flat.reshape(Ls, T, Z, Y, X, 4, 3)


def _mask(psi: np.ndarray, dims, par: int) -> np.ndarray:
    m = (parity(dims) == par)[..., None, None]
    return psi * m


# ----------------------------------------------------------------------------------------
# Even-odd preconditioned operator (Schur complement on even sites).
# ----------------------------------------------------------------------------------------
def mpc(U: np.ndarray, xe: np.ndarray, p: DWFParams) -> np.ndarray:
    """Mpc x = M5op x - 1/4 Dh_eo D+ M5op^-1 Dh_oe D+ x  on even-half vectors."""
    d = p.dims
    x = from_half(xe, d, 0)
    h = _mask(hop(U, s_apply(dplus_matrices(p), x)), d, 1)             # Dh_oe D+ x
    t = s_apply(dplus_matrices(p), s_apply(m5op_inv_matrices(p), h))   # D+ M5op^-1 (.)
    g = _mask(hop(U, t), d, 0)                                         # Dh_eo (.)
    y = s_apply(m5op_matrices(p), x) - 0.25 * g
    return to_half(y, d, 0)


def mpc_dag(U: np.ndarray, ye: np.ndarray, p: DWFParams) -> np.ndarray:
    """Mpc^dag y = M5op^dag y - 1/4 D+^dag Dh^dag_eo M5op^-dag D+^dag Dh^dag_oe y."""
    d = p.dims
    y = from_half(ye, d, 0)
    dpt = transpose_chi(dplus_matrices(p))
    h = _mask(hop(U, y, dag=True), d, 1)
    t = s_apply(transpose_chi(m5op_inv_matrices(p)), s_apply(dpt, h))
    g = _mask(hop(U, t, dag=True), d, 0)
    z = s_apply(transpose_chi(m5op_matrices(p)), y) - 0.25 * s_apply(dpt, g)
    return to_half(z, d, 0)


def mdagm(U: np.ndarray, xe: np.ndarray, p: DWFParams) -> np.ndarray:
    """A x = Mpc^dag Mpc x (Eq. 3 on the even sites)."""
    return mpc_dag(U, mpc(U, xe, p), p)


def even_site_coords(dims) -> np.ndarray:
    """(t, z, y, x) of the even sites, in the order of the even-half vectors."""
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X),
                             indexing="ij")
    c = np.stack([t, z, y, x], -1).reshape(-1, 4)
    return c[parity(dims).reshape(-1) == 0]


def mpc_at_sites(U: np.ndarray, xe: np.ndarray, p: DWFParams, sites, dag: bool = False):
    """(Mpc x) or (Mpc^dag x) at the even-half indices `sites`, evaluated site by site from the
    same definitions as mpc / mpc_dag: for an even site e, the odd intermediate at each of its
    eight neighbours o is built from the even neighbours of o, then the hop back to e.  For
    checks on lattices too large for the whole-lattice functions.  Returns (Ls, n, 4, 3)."""
    X, Y, Z, T = p.dims
    ext = np.array([T, Z, Y, X])
    half = -np.ones((T, Z, Y, X), dtype=np.int64)
    ec = even_site_coords(p.dims)
    half[tuple(ec.T)] = np.arange(len(ec))
    dp, m5, m5i = dplus_matrices(p), m5op_matrices(p), m5op_inv_matrices(p)
    if dag:
        dp, m5, m5i = transpose_chi(dp), transpose_chi(m5), transpose_chi(m5i)
    sgn = 1.0 if dag else -1.0

    def step(c, mu, d):            # neighbour c + d mu_hat, periodic (c = (t, z, y, x))
        n = np.array(c)
        n[3 - mu] = (n[3 - mu] + d) % ext[3 - mu]
        return tuple(n)

    def hop_at(get, c):            # (Dh psi)(c) or (Dh^dag psi)(c), psi(c') = get(c')
        out = np.zeros((p.Ls, 4, 3), dtype=complex)
        for mu in range(4):
            f, b = step(c, mu, +1), step(c, mu, -1)
            fwd = np.einsum("ab,lsb->lsa", U[c][mu], get(f))
            bwd = np.einsum("ab,lsb->lsa", dagger(U[b][mu]), get(b))
            out += np.einsum("ab,lbc->lac", ID4 + sgn * GAMMA[mu], fwd)
            out += np.einsum("ab,lbc->lac", ID4 - sgn * GAMMA[mu], bwd)
        return out

    x_at = lambda c: xe[:, half[c]]
    inner = {}

    def t_at(o):                   # the odd intermediate of the Schur complement at o
        if o not in inner:
            if not dag:            # D+ M5op^-1 Dh_oe D+ x
                inner[o] = s_apply(dp, s_apply(m5i, hop_at(lambda e: s_apply(dp, x_at(e)), o)))
            else:                  # M5op^-dag D+^dag Dh^dag_oe y
                inner[o] = s_apply(m5i, s_apply(dp, hop_at(x_at, o)))
        return inner[o]

    out = []
    for k in sites:
        e = tuple(ec[k])
        g = hop_at(t_at, e)
        if dag:
            g = s_apply(dp, g)     # D+^dag Dh^dag_eo (.)
        out.append(s_apply(m5, x_at(e)) - 0.25 * g)
    return np.stack(out, axis=1)


def m_eo(U: np.ndarray, xo_full: np.ndarray, p: DWFParams) -> np.ndarray:
    """M_eo x_o = -1/2 Dh_eo D+ x_o, as a full-lattice field (even sites)."""
    return _mask(-0.5 * hop(U, s_apply(dplus_matrices(p), xo_full)), p.dims, 0)


def m_oe(U: np.ndarray, xe_full: np.ndarray, p: DWFParams) -> np.ndarray:
    return _mask(-0.5 * hop(U, s_apply(dplus_matrices(p), xe_full)), p.dims, 1)


def eo_prepare(U: np.ndarray, b_full: np.ndarray, p: DWFParams) -> np.ndarray:
    """Even-site right-hand side of the Schur system: b_e - M_eo M5op^-1 b_o."""
    bo = _mask(b_full, p.dims, 1)
    be = _mask(b_full, p.dims, 0)
    rhs = be - m_eo(U, s_apply(m5op_inv_matrices(p), bo), p)
    return to_half(rhs, p.dims, 0)


def eo_reconstruct(U: np.ndarray, xe: np.ndarray, b_full: np.ndarray,
                   p: DWFParams) -> np.ndarray:
    """Full solution from the even part: x_o = M5op^-1 (b_o - M_oe x_e)."""
    x_e = from_half(xe, p.dims, 0)
    bo = _mask(b_full, p.dims, 1)
    xo = s_apply(m5op_inv_matrices(p), bo - m_oe(U, x_e, p))
    return x_e + _mask(xo, p.dims, 1)


# ----------------------------------------------------------------------------------------
# Blocks (the paper's node subdomains, Sec. 2.1 Eq. 1 and Sec. 2.3 Eq. 5).
# ----------------------------------------------------------------------------------------
def block_index(dims, block) -> np.ndarray:
    """Block id of every site on the (T,Z,Y,X) grid; blocks enumerated x fastest."""
    X, Y, Z, T = dims
    bx, by, bz, bt = block
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X),
                             indexing="ij")
    nx, ny, nz = X // bx, Y // by, Z // bz
    return (x // bx) + nx * ((y // by) + ny * ((z // bz) + nz * (t // bt)))


def block_links(U: np.ndarray, dims, block) -> np.ndarray:
    """Copy of U with every link whose two ends lie in different blocks set to zero."""
    bid = block_index(dims, block)
    Ub = U.copy()
    for mu in range(4):
        nb = np.roll(bid, -1, axis=3 - mu)           # block of x + mu
        Ub[..., mu, :, :] *= (nb == bid)[..., None, None]
    return Ub


def even_block_ids(dims, block) -> np.ndarray:
    return block_index(dims, block).reshape(-1)[parity(dims).reshape(-1) == 0]


def block_dot(a: np.ndarray, b: np.ndarray, eb: np.ndarray, nblocks: int) -> np.ndarray:
    """Per-block <a, b> over even-half vectors (sum over s, spin, colour, block sites)."""
    per_site = np.einsum("lvsc,lvsc->v", np.conj(a), b)
    return np.bincount(eb, weights=per_site.real, minlength=nblocks) + \
        1j * np.bincount(eb, weights=per_site.imag, minlength=nblocks)


# ----------------------------------------------------------------------------------------
# Solvers.
# ----------------------------------------------------------------------------------------
def vdot(a: np.ndarray, b: np.ndarray) -> complex:
    return complex(np.vdot(a.reshape(-1), b.reshape(-1)))


def norm(a: np.ndarray) -> float:
    return float(np.sqrt(vdot(a, a).real))


def cg(apply_a, b: np.ndarray, tol: float, maxit: int, x0=None):
    """Textbook conjugate gradient (Hestenes-Stiefel) for Hermitian positive-definite A.

    Stops when ||r_k|| <= tol ||b|| (recursively updated residual).  Returns (x, iterations,
    residual history ||r_k||/||b||).
    """
    bnorm = norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_a(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = vdot(r, r).real
    hist = [np.sqrt(rr) / bnorm]
    k = 0
    while k < maxit and np.sqrt(rr) > tol * bnorm:
        ap = apply_a(p)
        alpha = rr / vdot(p, ap).real
        x = x + alpha * p
        r = r - alpha * ap
        rr_new = vdot(r, r).real
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        k += 1
        hist.append(np.sqrt(rr) / bnorm)
    return x, k, hist


def block_cg(apply_ablk, r: np.ndarray, eb: np.ndarray, nblocks: int, iters: int):
    """l plain CG iterations on every block at once, zero initial guess, block-local dots.

    apply_ablk must be block-diagonal (hopping across block faces removed), so this is the
    same as running CG separately on each block with dots restricted to that block.
    """
    def per_site(v):            # broadcast a per-block scalar to the even-half shape
        return v[eb][None, :, None, None]

    x = np.zeros_like(r)
    res = r.copy()
    p = r.copy()
    rr = block_dot(res, res, eb, nblocks).real
    for _ in range(iters):
        ap = apply_ablk(p)
        pap = block_dot(p, ap, eb, nblocks).real
        alpha = np.where(pap > 0, rr / np.where(pap > 0, pap, 1.0), 0.0)
        x = x + per_site(alpha) * p
        res = res - per_site(alpha) * ap
        rr_new = block_dot(res, res, eb, nblocks).real
        beta = np.where(rr > 0, rr_new / np.where(rr > 0, rr, 1.0), 0.0)
        p = res + per_site(beta) * p
        rr = rr_new
    return x


def exact_block_operator(U: np.ndarray, p: DWFParams, block):
    """A_s = P_s A P_s for every block at once: the block-diagonal part of A, which is what
    the preconditioner M of Sec. 2.3, Eq. 5 is made of.  Applied block by block: the vector is
    restricted to one block, A is applied, and the result is restricted to the same block."""
    eb = even_block_ids(p.dims, block)
    nblocks = int(np.prod([p.dims[i] // block[i] for i in range(4)]))
    masks = [(eb == s)[None, :, None, None] for s in range(nblocks)]

    def apply(v):
        out = np.zeros_like(v)
        for m in masks:
            out += m * mdagm(U, v * m, p)
        return out
    return apply


def mspcg(U: np.ndarray, b: np.ndarray, p: DWFParams, block, inner_iters: int, tol: float,
          maxit: int, flexible: bool = False, local_op: str = "drop"):
    """Multisplitting preconditioned CG (Sec. 2.3).

    Outer: preconditioned CG on A = Mpc^dag Mpc with z = M^-1 r, M = direct sum of the
    block operators A_s (Eq. 5), each inverted approximately by `inner_iters` local CG
    iterations from a zero guess (Eq. 4 with x = 0).  beta is Fletcher-Reeves
    <r',z'>/<r,z>; flexible=True uses Polak-Ribiere <z', r' - r>/<r,z>.
    local_op="drop": A_s = Mpc_s^dag Mpc_s with hopping across block faces removed;
    local_op="exact": A_s = P_s A P_s.
    Returns (x, outer iterations, residual history ||r_k||/||b||).
    """
    d = p.dims
    eb = even_block_ids(d, block)
    nblocks = int(np.prod([d[i] // block[i] for i in range(4)]))

    def apply_a(v):
        return mdagm(U, v, p)

    if local_op == "drop":
        Ub = block_links(U, d, block)

        def apply_blk(v):
            return mdagm(Ub, v, p)
    elif local_op == "exact":
        apply_blk = exact_block_operator(U, p, block)
    else:
        raise ValueError(local_op)

    def precond(r):
        return block_cg(apply_blk, r, eb, nblocks, inner_iters)

    bnorm = norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    z = precond(r)
    pdir = z.copy()
    rz = vdot(r, z).real
    hist = [1.0]
    k = 0
    while k < maxit and hist[-1] > tol:
        ap = apply_a(pdir)
        alpha = rz / vdot(pdir, ap).real
        x = x + alpha * pdir
        r_old = r
        r = r - alpha * ap
        k += 1
        hist.append(norm(r) / bnorm)
        if hist[-1] <= tol:
            break
        z = precond(r)
        rz_new = vdot(r, z).real
        beta = (vdot(z, r - r_old).real if flexible else rz_new) / rz
        pdir = z + beta * pdir
        rz = rz_new
    return x, k, hist


def block_colours(dims, block, ncolours: int) -> np.ndarray:
    """Colour of every block (blocks enumerated x fastest) for the Schwarz sweeps:
    ncolours = 1 one colour; 2 the checkerboard of blocks, (b_x + b_y + b_z + b_t) mod 2;
    16 the 2^4 checkerboard, sum_mu 2^mu (b_mu mod 2).  The block coordinates b_mu count
    blocks along direction mu."""
    nb = [dims[i] // block[i] for i in range(4)]
    ids = np.arange(int(np.prod(nb)))
    bc = [(ids // int(np.prod(nb[:m]))) % nb[m] for m in range(4)]
    if ncolours == 1:
        return np.zeros_like(ids)
    if ncolours == 2:
        return (bc[0] + bc[1] + bc[2] + bc[3]) % 2
    if ncolours == 16:
        return sum((bc[m] % 2) << m for m in range(4))
    raise ValueError(ncolours)


def ms_solve(U: np.ndarray, b: np.ndarray, p: DWFParams, block, inner_iters: int,
             ncolours: int, tol: float, maxit: int, local_op: str = "exact"):
    """Stationary block iterations on A x = b built from the local solves of Sec. 2.3.

    ncolours = 1: the multisplitting iteration of Sec. 2.1 (Eq. 2): every block solves its
    own equation with the current solution outside it as the boundary value, all blocks at
    once, i.e. x <- x + M^-1 (b - A x) with M the direct sum of the A_s (Eq. 5).
    ncolours = 2 or 16: the same local solves one colour of blocks at a time, the residual
    recomputed before each colour (multiplicative Schwarz: 2 colours is the black-white
    checkerboard of blocks of the alternating Schwarz method, 16 the 2^4 checkerboard).
    Each A_s^-1 is approximated by `inner_iters` local CG iterations from a zero guess
    (block_cg); local_op as in mspcg.  One sweep = all colours once.  Returns (x, sweeps,
    history of ||b - A x|| / ||b|| after each sweep, starting with 1 for x = 0).
    """
    d = p.dims
    eb = even_block_ids(d, block)
    nblocks = int(np.prod([d[i] // block[i] for i in range(4)]))
    col = block_colours(d, block, ncolours)[eb]
    if local_op == "drop":
        Ub = block_links(U, d, block)

        def apply_blk(v):
            return mdagm(Ub, v, p)
    else:
        apply_blk = exact_block_operator(U, p, block)
    bnorm = norm(b)
    x = np.zeros_like(b)
    hist = [1.0]
    k = 0
    while k < maxit and hist[-1] > tol:
        for c in range(ncolours):
            r = b - mdagm(U, x, p)
            mask = (col == c)[None, :, None, None]
            x = x + block_cg(apply_blk, r * mask, eb, nblocks, inner_iters)
        k += 1
        hist.append(norm(b - mdagm(U, x, p)) / bnorm)
    return x, k, hist


def true_residual(U: np.ndarray, x: np.ndarray, b: np.ndarray, p: DWFParams) -> float:
    return norm(b - mdagm(U, x, p)) / norm(b)


# ----------------------------------------------------------------------------------------
# Pseudofermion action and its gradient with respect to the links.
# ----------------------------------------------------------------------------------------
def action(U: np.ndarray, phi: np.ndarray, p: DWFParams, X: np.ndarray | None = None,
           tol: float = 1e-13, maxit: int = 100000) -> float:
    """S = phi^dag (Mpc^dag Mpc)^-1 phi, evaluated as Re(2 phi^dag X - X^dag A X), which
    equals S at the exact solution and has an error quadratic in the solve residual."""
    if X is None:
        X, _, _ = cg(lambda v: mdagm(U, v, p), phi, tol, maxit)
    return float((2.0 * vdot(phi, X) - vdot(X, mdagm(U, X, p))).real)


def _hop_link_gradient(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Gradient of Re <a, Dh b> with respect to every link, PyTorch complex convention
    (dL/dRe U + i dL/dIm U), shape (T,Z,Y,X,4,3,3).

    U_mu(x) enters Dh twice: (1 - gamma_mu) U_mu(x) b(x+mu) at output x and
    (1 + gamma_mu) U_mu(x)^dag b(x) at output x+mu.  For Re tr(M U) the gradient is M^dag,
    which gives the two spin-traced colour outer products below (summed over s).
    """
    out = []
    for mu in range(4):
        pa = spin_mul(ID4 - GAMMA[mu], a)                        # (1 - g) a(x)
        bf = shift(b, mu, +1, 2)                                 # b(x + mu)
        t1 = np.einsum("ltzyxsa,ltzyxsb->tzyxab", pa, np.conj(bf))
        qa = spin_mul(ID4 + GAMMA[mu], shift(a, mu, +1, 2))      # (1 + g) a(x + mu)
        t2 = np.einsum("ltzyxsa,ltzyxsb->tzyxab", b, np.conj(qa))
        out.append(t1 + t2)
    return np.stack(out, axis=4)


def force(U: np.ndarray, phi: np.ndarray, p: DWFParams, X: np.ndarray | None = None,
          tol: float = 1e-13, maxit: int = 100000) -> np.ndarray:
    """dS/dU for S = phi^dag A^-1 phi, A = Mpc^dag Mpc (PyTorch complex gradient convention).

    dS = -2 Re <Y, dMpc X> with X = A^-1 phi, Y = Mpc X, and
    dMpc = -1/4 (dDh_eo D+ M5op^-1 Dh_oe D+ + Dh_eo D+ M5op^-1 dDh_oe D+), so
    dS = 1/2 Re( <Y, dDh W> + <Z, dDh V> ) with
    V = D+ X (even), W = D+ M5op^-1 Dh_oe V (odd), Z = M5op^-dag D+^dag Dh^dag_oe Y (odd).
    """
    d = p.dims
    if X is None:
        X, _, _ = cg(lambda v: mdagm(U, v, p), phi, tol, maxit)
    Yh = mpc(U, X, p)
    Xf = from_half(X, d, 0)
    Yf = from_half(Yh, d, 0)
    V = s_apply(dplus_matrices(p), Xf)
    W = s_apply(dplus_matrices(p), s_apply(m5op_inv_matrices(p), _mask(hop(U, V), d, 1)))
    Zo = s_apply(transpose_chi(m5op_inv_matrices(p)),
                 s_apply(transpose_chi(dplus_matrices(p)), _mask(hop(U, Yf, dag=True), d, 1)))
    return 0.5 * (_hop_link_gradient(Yf, W) + _hop_link_gradient(Zo, V))


# ----------------------------------------------------------------------------------------
# Dense builders for tiny lattices (used by the tests' brute-force pins).
# ----------------------------------------------------------------------------------------
def dense(apply, n_in: int, shape_in) -> np.ndarray:
    """Dense matrix of a linear map by applying it to unit vectors."""
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in, dtype=complex)
        e[k] = 1.0
        cols.append(apply(e.reshape(shape_in)).reshape(-1))
    return np.array(cols).T


# ----------------------------------------------------------------------------------------
# Cost arithmetic (Sec. 4.1, Eqs. 6-7).
# ----------------------------------------------------------------------------------------
def t_cg(alpha: float, P: float = 1.0) -> float:
    """Plain CG cost: computation P plus communication alpha P (Eq. 6)."""
    return P + alpha * P


def t_mspcg(alpha: float, l: int, g: float, P: float = 1.0) -> float:
    """MSPCG cost: ((1 + l) P + alpha P) / g for l local iterations and g-fold fewer
    global iterations (Eq. 7)."""
    return ((1 + l) * P + alpha * P) / g
