"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: algebraic identities,
closed forms, brute-force dense linear algebra on tiny lattices, finite differences, or the
worked example printed in the paper.  A dropped term, wrong sign, wrong index or transposed
operand anywhere in the operator, the solvers or the force fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import dwf_oracle as o
from paper_1804_08593_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand5(rng, dims, Ls):
    X, Y, Z, T = dims
    s = (Ls, T, Z, Y, X, 4, 3)
    return rng.standard_normal(s) + 1j * rng.standard_normal(s)


def rand4(rng, dims):
    X, Y, Z, T = dims
    s = (T, Z, Y, X, 4, 3)
    return rng.standard_normal(s) + 1j * rng.standard_normal(s)


def randh(rng, dims, Ls):
    X, Y, Z, T = dims
    s = (Ls, X * Y * Z * T // 2, 4, 3)
    return rng.standard_normal(s) + 1j * rng.standard_normal(s)


def g5r5(psi):
    """(Gamma5 R5 psi)_s = gamma_5 psi_{Ls-1-s}."""
    return o.spin_mul(o.GAMMA5, psi[::-1])


SHAMIR = dict(M5=1.8, mf=0.1, b=1.0, c=0.0)
MOBIUS = dict(M5=1.8, mf=0.1, b=1.5, c=0.5)


# ------------------------------------------------------------------------------------------
# Gamma matrices.
# ------------------------------------------------------------------------------------------
def test_gamma_algebra():
    for m in range(4):
        assert np.allclose(o.GAMMA[m], o.GAMMA[m].conj().T)
        for n in range(4):
            anti = o.GAMMA[m] @ o.GAMMA[n] + o.GAMMA[n] @ o.GAMMA[m]
            assert np.allclose(anti, 2.0 * (m == n) * np.eye(4))
    assert np.allclose(o.GAMMA5, np.diag([1, 1, -1, -1]))
    for P in (o.P_PLUS, o.P_MINUS):
        assert np.allclose(P @ P, P)
    assert np.allclose(o.P_PLUS @ o.P_MINUS, 0)


# ------------------------------------------------------------------------------------------
# Wilson operator: free-field plane-wave closed form, adjoint, gamma5-hermiticity.
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 3), (3, 1, 1, 2), (2, 3, 0, 1)])
def test_free_wilson_plane_wave(n):
    """U = 1: D_W(-M5) e^{ipx} chi = e^{ipx} [4 - M5 - sum cos p + i sum gamma_mu sin p] chi."""
    dims = (4, 4, 6, 8)
    X, Y, Z, T = dims
    M5 = 1.8
    pmom = [2 * np.pi * n[m] / dims[m] for m in range(4)]
    rng = np.random.default_rng(0)
    chi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X),
                             indexing="ij")
    phase = np.exp(1j * (pmom[0] * x + pmom[1] * y + pmom[2] * z + pmom[3] * t))
    psi = phase[..., None, None] * chi
    out = o.wilson(inputs.unit_links(dims), psi, M5)
    mat = (4 - M5 - sum(np.cos(pmom))) * np.eye(4) + \
        1j * sum(o.GAMMA[m] * np.sin(pmom[m]) for m in range(4))
    expect = phase[..., None, None] * (mat @ chi)
    assert np.abs(out - expect).max() < 1e-13


def test_hop_adjoint_and_gamma5():
    rng = np.random.default_rng(1)
    dims = (4, 2, 4, 6)
    U = inputs.gauge_links(dims, 0.7, rng)
    a, b = rand5(rng, dims, 3), rand5(rng, dims, 3)
    lhs = o.vdot(a, o.hop(U, b))
    rhs = o.vdot(o.hop(U, a, dag=True), b)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # gamma5 Dh gamma5 = Dh^dag
    g5 = o.spin_mul(o.GAMMA5, o.hop(U, o.spin_mul(o.GAMMA5, b)))
    assert np.abs(g5 - o.hop(U, b, dag=True)).max() < 1e-12


# ------------------------------------------------------------------------------------------
# Gauge covariance: D[U^g](g psi) = g D[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag.
# ------------------------------------------------------------------------------------------
def gauge_rotate(U, g):
    Ug = np.empty_like(U)
    for mu in range(4):
        gfwd = np.roll(g, -1, axis=3 - mu)
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ o.dagger(gfwd)
    return Ug


def rot_field(g, psi):
    return np.einsum("tzyxab,...tzyxsb->...tzyxsa", g, psi)


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS])
def test_gauge_covariance(prm):
    rng = np.random.default_rng(2)
    dims = (4, 4, 2, 4)
    Ls = 4
    p = o.DWFParams(dims, Ls, **prm)
    U = inputs.gauge_links(dims, 0.5, rng)
    g = inputs.gauge_transform(dims, rng)
    Ug = gauge_rotate(U, g)
    psi = rand5(rng, dims, Ls)
    assert np.abs(o.dwf(Ug, rot_field(g, psi), p) - rot_field(g, o.dwf(U, psi, p))).max() < 1e-12
    # even-odd operator and its normal operator on even-half vectors
    xe = randh(rng, dims, Ls)
    full = o.from_half(xe, dims)
    gx = o.to_half(rot_field(g, full), dims)
    lhs = o.mdagm(Ug, gx, p)
    rhs = o.to_half(rot_field(g, o.from_half(o.mdagm(U, xe, p), dims)), dims)
    assert np.abs(lhs - rhs).max() < 1e-12


# ------------------------------------------------------------------------------------------
# Gamma5 R5 hermiticity and adjoints.
# ------------------------------------------------------------------------------------------
def test_gamma5_r5_hermiticity_shamir():
    """Shamir: D^dag = Gamma5 R5 D Gamma5 R5 (fixes the s-shift/projector pairing of K)."""
    rng = np.random.default_rng(3)
    dims = (4, 2, 2, 4)
    Ls = 6
    p = o.DWFParams(dims, Ls, **SHAMIR)
    U = inputs.gauge_links(dims, 0.6, rng)
    a, b = rand5(rng, dims, Ls), rand5(rng, dims, Ls)
    lhs = o.vdot(a, o.dwf(U, b, p))
    rhs = o.vdot(g5r5(o.dwf(U, g5r5(a), p)), b)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    assert np.abs(o.dwf(U, a, p, dag=True) - g5r5(o.dwf(U, g5r5(a), p))).max() < 1e-12


def test_gamma5_r5_hermiticity_mobius():
    """Moebius: (D D+^-1) is Gamma5 R5 hermitian while D itself is not."""
    rng = np.random.default_rng(4)
    dims = (4, 2, 2, 4)
    Ls = 6
    p = o.DWFParams(dims, Ls, **MOBIUS)
    U = inputs.gauge_links(dims, 0.6, rng)
    dpinv = np.array([np.linalg.inv(m) for m in o.dplus_matrices(p)])

    def dd(v):
        return o.dwf(U, o.s_apply(dpinv, v), p)

    a, b = rand5(rng, dims, Ls), rand5(rng, dims, Ls)
    lhs = o.vdot(a, dd(b))
    rhs = o.vdot(g5r5(dd(g5r5(a))), b)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    # negative control: the identity fails for D itself when c != 0
    l2 = o.vdot(a, o.dwf(U, b, p))
    r2 = o.vdot(g5r5(o.dwf(U, g5r5(a), p)), b)
    assert abs(l2 - r2) > 1e-3 * abs(l2)


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS])
def test_adjoints(prm):
    rng = np.random.default_rng(5)
    dims = (4, 4, 2, 2)
    Ls = 5
    p = o.DWFParams(dims, Ls, **prm)
    U = inputs.gauge_links(dims, 0.6, rng)
    a, b = rand5(rng, dims, Ls), rand5(rng, dims, Ls)
    assert abs(o.vdot(a, o.dwf(U, b, p)) - o.vdot(o.dwf(U, a, p, dag=True), b)) < 1e-10
    ae, be = randh(rng, dims, Ls), randh(rng, dims, Ls)
    lhs = o.vdot(ae, o.mpc(U, be, p))
    rhs = o.vdot(o.mpc_dag(U, ae, p), be)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


# ------------------------------------------------------------------------------------------
# Fifth dimension: M5op inverse against the Shamir geometric closed form.
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("Ls", [4, 8, 12, 16])
def test_m5op_inverse_shamir_closed_form(Ls):
    """Shamir M5op = (5 - M5) - K.  With a = 5 - M5 and S the wrapped shift (S^Ls = -mf),
    (a - S)^-1 = sum_{k<Ls} S^k a^{-k-1} / (1 + mf a^-Ls)."""
    M5, mf = 1.8, 0.05
    p = o.DWFParams((2, 2, 2, 2), Ls, M5, mf)
    inv = o.m5op_inv_matrices(p)
    a = 5 - M5
    den = 1 + mf * a ** (-Ls)
    ref = np.zeros((2, Ls, Ls))
    for s in range(Ls):
        for t in range(Ls):
            # P+ rows: K moves s-1 -> s; P- rows: K moves s+1 -> s
            k = (s - t) % Ls
            ref[0, s, t] = a ** (-1 - k) * (1.0 if s >= t else -mf) / den
            k = (t - s) % Ls
            ref[1, s, t] = a ** (-1 - k) * (1.0 if t >= s else -mf) / den
    assert np.abs(inv - ref).max() < 1e-15
    m = o.m5op_matrices(p)
    for c in range(2):
        assert np.abs(m[c] @ inv[c] - np.eye(Ls)).max() < 1e-15


def test_m5op_inverse_mobius():
    p = o.DWFParams((2, 2, 2, 2), 12, 1.8, 0.005, 1.5, 0.5)
    m, inv = o.m5op_matrices(p), o.m5op_inv_matrices(p)
    for c in range(2):
        assert np.abs(m[c] @ inv[c] - np.eye(12)).max() < 1e-14


# ------------------------------------------------------------------------------------------
# Domain-wall determinant identity: det D(mf) / det D(1) = det D_eff(mf),
# D_eff = (1+mf)/2 + (1-mf)/2 gamma5 eps_Ls(H),  H = gamma5 (b+c) D_W / (2 + (b-c) D_W),
# eps_Ls(H) = [(1+H)^Ls - (1-H)^Ls] / [(1+H)^Ls + (1-H)^Ls].
# This is the standard transfer-matrix result for Moebius domain-wall fermions; it fixes the
# mass corners of K, the roles of b and c and the sign of M5 all at once.
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prm", [dict(b=1.0, c=0.0, mf=0.1), dict(b=1.5, c=0.5, mf=0.07)])
def test_dwf_determinant_identity(prm):
    rng = np.random.default_rng(7)
    dims = (2, 2, 2, 2)
    X, Y, Z, T = dims
    V = X * Y * Z * T
    Ls, M5 = 4, 1.8
    U = inputs.gauge_links(dims, 0.5, rng)
    shape = (Ls, T, Z, Y, X, 4, 3)

    def logdet(mf):
        pm = o.DWFParams(dims, Ls, M5, mf, prm["b"], prm["c"])
        return np.linalg.slogdet(o.dense(lambda v: o.dwf(U, v, pm), Ls * V * 12, shape))

    s_m, s_1 = logdet(prm["mf"]), logdet(1.0)
    ratio = s_m[0] / s_1[0] * np.exp(s_m[1] - s_1[1])
    DW = o.dense(lambda v: o.wilson(U, v, M5), V * 12, (T, Z, Y, X, 4, 3))
    G5 = np.kron(np.eye(V), np.kron(o.GAMMA5, np.eye(3)))
    b, c, mf = prm["b"], prm["c"], prm["mf"]
    H = G5 @ ((b + c) * DW) @ np.linalg.inv(2 * np.eye(V * 12) + (b - c) * DW)
    H = 0.5 * (H + H.conj().T)
    lam, W = np.linalg.eigh(H)
    eps = ((1 + lam) ** Ls - (1 - lam) ** Ls) / ((1 + lam) ** Ls + (1 - lam) ** Ls)
    Deff = (1 + mf) / 2 * np.eye(V * 12) + (1 - mf) / 2 * G5 @ ((W * eps) @ W.conj().T)
    sd = np.linalg.slogdet(Deff)
    deff = sd[0] * np.exp(sd[1])
    assert abs(ratio - deff) < 1e-9 * abs(deff)


# ------------------------------------------------------------------------------------------
# Even-odd Schur complement against a dense solve of the full operator.
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS])
def test_schur_consistency(prm):
    rng = np.random.default_rng(8)
    dims = (2, 2, 2, 2)
    X, Y, Z, T = dims
    V = X * Y * Z * T
    Ls = 4
    p = o.DWFParams(dims, Ls, **prm)
    U = inputs.gauge_links(dims, 0.5, rng)
    shape = (Ls, T, Z, Y, X, 4, 3)
    D = o.dense(lambda v: o.dwf(U, v, p), Ls * V * 12, shape)
    bfull = rand5(rng, dims, Ls)
    x = np.linalg.solve(D, bfull.reshape(-1)).reshape(shape)
    nh = Ls * (V // 2) * 12
    Mpc = o.dense(lambda v: o.mpc(U, v, p), nh, (Ls, V // 2, 4, 3))
    rhs = o.eo_prepare(U, bfull, p)
    xe = np.linalg.solve(Mpc, rhs.reshape(-1)).reshape(Ls, V // 2, 4, 3)
    assert np.abs(xe - o.to_half(x, dims)).max() < 1e-12 * np.abs(x).max()
    assert np.abs(o.eo_reconstruct(U, xe, bfull, p) - x).max() < 1e-12 * np.abs(x).max()


def test_normal_operator_hpd_and_second_neighbour():
    """A = Mpc^dag Mpc is Hermitian positive definite; D^dag D reaches second neighbours
    (Sec. 2.2) while D reaches only first neighbours."""
    rng = np.random.default_rng(9)
    dims = (4, 2, 2, 2)
    Ls = 2
    p = o.DWFParams(dims, Ls, **MOBIUS)
    U = inputs.gauge_links(dims, 0.5, rng)
    nh = Ls * 16 * 12
    A = o.dense(lambda v: o.mdagm(U, v, p), nh, (Ls, 16, 4, 3))
    assert np.abs(A - A.conj().T).max() < 1e-12
    assert np.linalg.eigvalsh(A).min() > 0
    # point source at the origin: D reaches only nearest neighbours, D^dag D also the
    # diagonal second neighbours x + mu + nu; straight two-hop paths cancel because
    # (1 + gamma_mu)(1 - gamma_mu) = 0.
    dims2 = (4, 4, 2, 2)
    U2 = inputs.gauge_links(dims2, 0.5, rng)
    X, Y, Z, T = dims2
    psi = np.zeros((Ls, T, Z, Y, X, 4, 3), dtype=complex)
    psi[0, 0, 0, 0, 0, 0, 0] = 1.0
    p2 = o.DWFParams(dims2, Ls, **MOBIUS)
    d1 = np.abs(o.dwf(U2, psi, p2)).sum(axis=(0, 5, 6))
    d2 = np.abs(o.dwf(U2, o.dwf(U2, psi, p2), p2, dag=True)).sum(axis=(0, 5, 6))
    assert d1[0, 0, 0, 1] > 0 and d1[0, 0, 1, 1] == 0 and d1[0, 0, 0, 2] == 0
    assert d2[0, 0, 1, 1] > 0 and d2[0, 0, 2, 0] == 0 and d2[0, 0, 0, 2] == 0


# ------------------------------------------------------------------------------------------
# Solvers against brute-force dense solves.
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS])
def test_cg_matches_dense_solve(prm):
    rng = np.random.default_rng(10)
    dims = (2, 2, 2, 2)
    Ls = 4
    p = o.DWFParams(dims, Ls, **prm)
    U = inputs.gauge_links(dims, 0.4, rng)
    phi = inputs.even_source(dims, Ls, rng)
    nh = phi.size
    A = o.dense(lambda v: o.mdagm(U, v, p), nh, phi.shape)
    xd = np.linalg.solve(A, phi.reshape(-1))
    x, k, hist = o.cg(lambda v: o.mdagm(U, v, p), phi, 1e-13, 1000)
    assert hist[-1] <= 1e-13
    assert np.abs(x.reshape(-1) - xd).max() < 1e-11 * np.abs(xd).max()
    assert o.true_residual(U, x, phi, p) < 1e-12
    # non-zero initial guess is a restart
    x2, k2, _ = o.cg(lambda v: o.mdagm(U, v, p), phi, 1e-13, 1000, x0=0.5 * x)
    assert np.abs(x2.reshape(-1) - xd).max() < 1e-11 * np.abs(xd).max()


def test_cg_iteration_bound_on_tiny_problem():
    """CG terminates in at most n steps on an n-dimensional HPD system (exact arithmetic);
    on a well conditioned 2^4 x Ls=2 problem it converges long before n = 192."""
    rng = np.random.default_rng(11)
    dims = (2, 2, 2, 2)
    p = o.DWFParams(dims, 2, 1.8, 0.5)
    U = inputs.gauge_links(dims, 0.3, rng)
    phi = inputs.even_source(dims, 2, rng)
    _, k, hist = o.cg(lambda v: o.mdagm(U, v, p), phi, 1e-12, 1000)
    assert k <= phi.size and hist[-1] <= 1e-12


# ------------------------------------------------------------------------------------------
# Multisplitting preconditioner (Sec. 2.3, Eqs. 4-5).
# ------------------------------------------------------------------------------------------
def test_blocked_operator_is_block_diagonal():
    rng = np.random.default_rng(12)
    dims = (4, 4, 4, 4)
    block = (2, 2, 2, 2)
    Ls = 2
    p = o.DWFParams(dims, Ls, **MOBIUS)
    U = inputs.gauge_links(dims, 0.5, rng)
    Ub = o.block_links(U, dims, block)
    eb = o.even_block_ids(dims, block)
    v = randh(rng, dims, Ls)
    for blk in (0, 5, 15):
        vb = v * (eb == blk)[None, :, None, None]
        out = o.mdagm(Ub, vb, p)
        assert np.abs(out[:, eb != blk]).max() == 0.0
        assert np.abs(out[:, eb == blk]).max() > 0.0
    # every link with both ends in one block is kept, the others are zero
    bid = o.block_index(dims, block)
    for mu in range(4):
        same = np.roll(bid, -1, axis=3 - mu) == bid
        assert np.all(Ub[..., mu, :, :][same] == U[..., mu, :, :][same])
        assert np.all(Ub[..., mu, :, :][~same] == 0)


def test_block_local_operator_vs_exact_block():
    """P_s A P_s (the block-diagonal part of A, Eq. 5) and the dropped-hop block
    operator differ only on sites next to a block face (the second-neighbour terms of D^dag D,
    Sec. 2.2); both are Hermitian positive definite (Sec. 2.3)."""
    rng = np.random.default_rng(13)
    dims = (4, 2, 2, 2)
    block = (2, 2, 2, 2)
    Ls = 2
    p = o.DWFParams(dims, Ls, **SHAMIR)
    U = inputs.gauge_links(dims, 0.5, rng)
    Ub = o.block_links(U, dims, block)
    eb = o.even_block_ids(dims, block)
    shape = (Ls, 16, 4, 3)
    n = Ls * 16 * 12
    A = o.dense(lambda v: o.mdagm(U, v, p), n, shape)
    Ad = o.dense(lambda v: o.mdagm(Ub, v, p), n, shape)
    site_of = np.broadcast_to(np.arange(16)[None, :, None, None], shape).reshape(-1)
    blk = eb[site_of]
    PAP = A * (blk[:, None] == blk[None, :])
    for M in (PAP, Ad):
        assert np.abs(M - M.conj().T).max() < 1e-12
        assert np.linalg.eigvalsh(M).min() > 0
    assert np.abs(PAP - Ad).max() > 1e-3   # they are different operators


def test_block_cg_equals_separate_block_solves():
    rng = np.random.default_rng(14)
    dims = (4, 4, 2, 2)
    block = (2, 2, 2, 2)
    Ls = 3
    p = o.DWFParams(dims, Ls, **MOBIUS)
    U = inputs.gauge_links(dims, 0.5, rng)
    Ub = o.block_links(U, dims, block)
    eb = o.even_block_ids(dims, block)
    nb = 4
    r = randh(rng, dims, Ls)
    z = o.block_cg(lambda v: o.mdagm(Ub, v, p), r, eb, nb, 4)
    ref = np.zeros_like(r)
    for blk in range(nb):
        m = (eb == blk)[None, :, None, None]
        xb, _, _ = o.cg(lambda v: o.mdagm(Ub, v, p), r * m, 0.0, 4)
        ref += xb * m
    assert np.abs(z - ref).max() < 1e-12 * np.abs(ref).max()


def test_block_cg_one_iteration_closed_form():
    """One local CG step from zero: z_s = (<r_s, r_s> / <r_s, A_s r_s>) r_s."""
    rng = np.random.default_rng(15)
    dims = (4, 4, 2, 2)
    block = (2, 2, 2, 2)
    Ls = 2
    p = o.DWFParams(dims, Ls, **SHAMIR)
    U = inputs.gauge_links(dims, 0.5, rng)
    Ub = o.block_links(U, dims, block)
    eb = o.even_block_ids(dims, block)
    r = randh(rng, dims, Ls)
    z = o.block_cg(lambda v: o.mdagm(Ub, v, p), r, eb, 4, 1)
    Ar = o.mdagm(Ub, r, p)
    for blk in range(4):
        m = eb == blk
        coef = np.vdot(r[:, m], r[:, m]).real / np.vdot(r[:, m], Ar[:, m]).real
        assert np.abs(z[:, m] - coef * r[:, m]).max() < 1e-13 * np.abs(r).max()


def test_mspcg_solution_and_exact_preconditioner():
    rng = np.random.default_rng(16)
    dims = (4, 2, 2, 2)
    Ls = 4
    p = o.DWFParams(dims, Ls, 1.8, 0.5, 1.5, 0.5)
    U = inputs.gauge_links(dims, 0.4, rng)
    phi = inputs.even_source(dims, Ls, rng)
    A = o.dense(lambda v: o.mdagm(U, v, p), phi.size, phi.shape)
    xd = np.linalg.solve(A, phi.reshape(-1))
    for lop in ("drop", "exact"):
        for flex in (False, True):
            x, k, hist = o.mspcg(U, phi, p, (2, 2, 2, 2), 3, 1e-12, 300, flexible=flex,
                                 local_op=lop)
            assert hist[-1] <= 1e-12, (lop, flex)
            assert np.abs(x.reshape(-1) - xd).max() < 1e-10 * np.abs(xd).max()
    # one block = the whole lattice, many local iterations: M^-1 ~ A^-1, so the outer
    # iteration finishes in very few steps
    _, k1, h1 = o.mspcg(U, phi, p, dims, 400, 1e-10, 50)
    assert k1 <= 2 and h1[-1] <= 1e-10


def test_exact_block_operator_is_the_diagonal_block_of_A():
    """local_op='exact' applies P_s A P_s: its dense matrix equals A with every entry that
    couples two different blocks set to zero (Sec. 2.3, Eq. 5 and its figure)."""
    rng = np.random.default_rng(20)
    dims = (4, 2, 2, 2)
    Ls = 2
    p = o.DWFParams(dims, Ls, **MOBIUS)
    U = inputs.gauge_links(dims, 0.5, rng)
    shape = (Ls, 16, 4, 3)
    n = Ls * 16 * 12
    A = o.dense(lambda v: o.mdagm(U, v, p), n, shape)
    M = o.dense(o.exact_block_operator(U, p, (2, 2, 2, 2)), n, shape)
    eb = o.even_block_ids(dims, (2, 2, 2, 2))
    blk = eb[np.broadcast_to(np.arange(16)[None, :, None, None], shape).reshape(-1)]
    same = blk[:, None] == blk[None, :]
    assert np.abs(M - A * same).max() == 0.0
    assert np.abs(A * ~same).max() > 0.0


def test_mspcg_reduces_global_iterations():
    """Direction of the paper's result (Sec. 3): with the block-diagonal part of A as the
    preconditioner, fewer global iterations than plain CG."""
    rng = np.random.default_rng(3)
    dims, Ls = (8, 4, 2, 2), 4
    p = o.DWFParams(dims, Ls, 1.8, 0.1, 1.0, 0.0)
    U = inputs.gauge_links(dims, 0.2, rng)
    phi = inputs.even_source(dims, Ls, rng)
    _, kcg, _ = o.cg(lambda v: o.mdagm(U, v, p), phi, 1e-10, 5000)
    x, kex, hist = o.mspcg(U, phi, p, (4, 4, 2, 2), 6, 1e-10, 5000, local_op="exact")
    assert hist[-1] <= 1e-10
    assert o.true_residual(U, x, phi, p) < 1e-9
    assert kex < kcg
    _, kdr, _ = o.mspcg(U, phi, p, (4, 4, 2, 2), 6, 1e-10, 5000, local_op="drop")
    assert kdr < kcg


# ------------------------------------------------------------------------------------------
# Stationary block iterations: the multisplitting iteration (Sec. 2.1, Eq. 2) and the
# multiplicative Schwarz sweeps over 2- and 16-colour checkerboards of blocks.
# ------------------------------------------------------------------------------------------
def test_block_colours_separate_neighbouring_blocks():
    """2 colours: blocks that share a face differ; 16 colours: blocks that differ by one step in
    any set of directions differ (faces, edges, corners), blocks two steps apart agree; every
    colour class has the same size."""
    dims, block = (8, 8, 4, 4), (2, 2, 2, 2)
    nb = [4, 4, 2, 2]
    ids = np.arange(int(np.prod(nb)))
    bc = np.stack([(ids // int(np.prod(nb[:m]))) % nb[m] for m in range(4)], 1)

    def bid(c):
        c = [c[m] % nb[m] for m in range(4)]
        return c[0] + nb[0] * (c[1] + nb[1] * (c[2] + nb[2] * c[3]))
    assert np.all(o.block_colours(dims, block, 1) == 0)
    c2 = o.block_colours(dims, block, 2)
    c16 = o.block_colours(dims, block, 16)
    assert sorted(np.bincount(c2)) == [32, 32] and sorted(np.bincount(c16)) == [4] * 16
    for i in ids:
        for mu in range(4):
            for sgn in (1, -1):
                n = bc[i].copy()
                n[mu] += sgn
                assert c2[bid(n)] != c2[i]
        for step in range(1, 16):   # every nonempty set of directions
            n = bc[i] + np.array([(step >> m) & 1 for m in range(4)])
            assert c16[bid(n)] != c16[i]
        n = bc[i].copy()
        n[0] += 2
        assert c16[bid(n)] == c16[i] and c2[bid(n)] == c2[i]


def test_ms_sweeps_are_block_jacobi_and_block_gauss_seidel():
    """With exact local solves, one sweep of the multisplitting iteration is block Jacobi,
    x <- x + D^-1 (b - A x) with D the block-diagonal part of A (Eqs. 2 and 5), and the
    2-colour sweep is block Gauss-Seidel over the colours; checked against dense algebra on
    2^4 blocks of a 4x2x2x2 x 4 lattice (two blocks)."""
    rng = np.random.default_rng(31)
    dims, Ls, block = (4, 2, 2, 2), 4, (2, 2, 2, 2)
    p = o.DWFParams(dims, Ls, 1.8, 0.5, 1.5, 0.5)
    U = inputs.gauge_links(dims, 0.3, rng)
    phi = inputs.even_source(dims, Ls, rng)
    n = phi.size
    A = o.dense(lambda v: o.mdagm(U, v, p), n, phi.shape)
    eb = o.even_block_ids(dims, block)
    comp_blk = np.broadcast_to(eb[None, :, None, None], phi.shape).reshape(-1)
    D = A * (comp_blk[:, None] == comp_blk[None, :])
    b = phi.reshape(-1)
    # multisplitting iteration (additive): two sweeps
    x, k, hist = o.ms_solve(U, phi, p, block, 400, 1, 0.0, 2)
    x1 = np.linalg.solve(D, b)
    x2 = x1 + np.linalg.solve(D, b - A @ x1)
    assert k == 2
    assert np.abs(x.reshape(-1) - x2).max() < 1e-9 * np.abs(x2).max()
    assert abs(hist[1] - np.linalg.norm(b - A @ x1) / np.linalg.norm(b)) < 1e-9
    # 2 colours (block 0 then block 1), one sweep
    x, _, _ = o.ms_solve(U, phi, p, block, 400, 2, 0.0, 1)
    col = o.block_colours(dims, block, 2)[comp_blk]
    xd = np.zeros(n, complex)
    for c in range(2):
        m = col == c
        r = b - A @ xd
        xd[m] += np.linalg.solve(A[np.ix_(m, m)], r[m])
    assert np.abs(x.reshape(-1) - xd).max() < 1e-9 * np.abs(xd).max()
    # 16 colours with one block per colour bit 0 (two blocks along x): the same sweep
    x16, _, _ = o.ms_solve(U, phi, p, block, 400, 16, 0.0, 1)
    assert np.abs(x16 - x).max() < 1e-12 * np.abs(x).max()


def test_ms_one_block_many_local_iterations_solves_at_once():
    """One block = the whole lattice with many local iterations: M^-1 ~ A^-1, so one sweep of
    the multisplitting iteration reaches a small residual."""
    rng = np.random.default_rng(32)
    dims, Ls = (4, 2, 2, 2), 4
    p = o.DWFParams(dims, Ls, 1.8, 0.3, 1.0, 0.0)
    U = inputs.gauge_links(dims, 0.3, rng)
    phi = inputs.even_source(dims, Ls, rng)
    _, k, hist = o.ms_solve(U, phi, p, dims, 400, 1, 1e-9, 5)
    assert k == 1 and hist[1] <= 1e-9


# ------------------------------------------------------------------------------------------
# Force: central finite differences of the action, and the gradient convention.
# ------------------------------------------------------------------------------------------
def test_gradient_convention_matches_torch():
    """For real L, the gradient is dL/dRe U + i dL/dIm U (PyTorch's convention): for
    L = Re tr(M U) it is M^dag; for L = |z|^2 it is 2z."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(17)
    M = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    U = torch.tensor(rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)),
                     requires_grad=True)
    L = torch.real(torch.trace(torch.tensor(M) @ U))
    L.backward()
    assert np.abs(U.grad.numpy() - M.conj().T).max() < 1e-14
    z = torch.tensor(1.5 - 0.7j, dtype=torch.complex128, requires_grad=True)
    (z.abs() ** 2).backward()
    assert abs(complex(z.grad) - 2 * (1.5 - 0.7j)) < 1e-14


@pytest.mark.parametrize("prm", [SHAMIR, MOBIUS])
def test_force_matches_central_differences(prm):
    rng = np.random.default_rng(18)
    dims = (2, 2, 2, 4)
    Ls = 4
    p = o.DWFParams(dims, Ls, **prm)
    U = inputs.gauge_links(dims, 0.5, rng)
    phi = inputs.even_source(dims, Ls, rng)

    def S(Uv):
        A = o.dense(lambda v: o.mdagm(Uv, v, p), phi.size, phi.shape)
        return float(np.vdot(phi.reshape(-1), np.linalg.solve(A, phi.reshape(-1))).real)

    F = o.force(U, phi, p, tol=1e-14)
    h = 1e-5
    for k in range(3):
        Om = inputs.su3_directions(dims, rng)
        lam, Vv = np.linalg.eigh(Om)

        def rot(hh):
            e = (Vv * np.exp(1j * hh * lam)[..., None, :]) @ o.dagger(Vv)
            return e @ U

        fd = (S(rot(h)) - S(rot(-h))) / (2 * h)
        # dS/dh = sum Re tr(F^dag dU/dh), dU/dh = i Omega U
        an = float(np.sum(np.real(np.conj(F) * (1j * Om @ U))))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


def test_force_gauge_covariance():
    """Under U -> U^g, phi -> g phi the action is invariant and
    dS/dU_mu(x) -> g(x) dS/dU_mu(x) g(x+mu)^dag (from dU^g = g(x) dU g(x+mu)^dag)."""
    rng = np.random.default_rng(19)
    dims = (2, 2, 2, 4)
    Ls = 3
    p = o.DWFParams(dims, Ls, **MOBIUS)
    U = inputs.gauge_links(dims, 0.5, rng)
    phi = inputs.even_source(dims, Ls, rng)
    g = inputs.gauge_transform(dims, rng)
    F = o.force(U, phi, p, tol=1e-14)
    gphi = o.to_half(rot_field(g, o.from_half(phi, dims)), dims)
    Fg = o.force(gauge_rotate(U, g), gphi, p, tol=1e-14)
    for mu in range(4):
        gf = np.roll(g, -1, axis=3 - mu)
        expect = g @ F[..., mu, :, :] @ o.dagger(gf)
        assert np.abs(Fg[..., mu, :, :] - expect).max() < 1e-9 * np.abs(F).max()


# ------------------------------------------------------------------------------------------
# Cost arithmetic: the worked example of Sec. 4.1.
# ------------------------------------------------------------------------------------------
def test_cost_model_worked_example():
    vals = {}
    with open(os.path.join(GOLDEN, "cost_model.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    ratio = o.t_cg(vals["alpha"]) / o.t_mspcg(vals["alpha"], int(vals["l"]), vals["g"])
    assert abs(ratio - vals["speedup_exact"]) < 1e-15
    assert round(ratio) == vals["speedup_quoted"]
    assert o.t_cg(0.0) == 1.0 and o.t_mspcg(0.0, 0, 1.0) == 1.0


def test_action_estimator_against_dense_solve():
    """S = Re(2 phi^dag X - X^dag A X) equals phi^dag A^-1 phi at the exact solution and its
    error is quadratic in the solution error."""
    rng = np.random.default_rng(22)
    dims, Ls = (2, 2, 2, 2), 4
    p = o.DWFParams(dims, Ls, **MOBIUS)
    U = inputs.gauge_links(dims, 0.5, rng)
    phi = inputs.even_source(dims, Ls, rng)
    A = o.dense(lambda v: o.mdagm(U, v, p), phi.size, phi.shape)
    x = np.linalg.solve(A, phi.reshape(-1))
    S = float(np.vdot(phi.reshape(-1), x).real)
    assert abs(o.action(U, phi, p, X=x.reshape(phi.shape)) - S) < 1e-12 * abs(S)
    e = 1e-4 * (rng.standard_normal(x.shape) + 1j * rng.standard_normal(x.shape))
    err = abs(o.action(U, phi, p, X=(x + e).reshape(phi.shape)) - S)
    assert err <= 1.01 * float(np.vdot(e, A @ e).real) + 1e-12


@pytest.mark.parametrize("dims,b,c", [((4, 4, 2, 4), 1.5, 0.5), ((2, 4, 4, 2), 1.0, 0.0)])
def test_site_sampled_mpc_equals_whole_lattice(dims, b, c):
    """mpc_at_sites (used to check full-size lattices at sampled sites) restates Mpc and
    Mpc^dag site by site; it must agree with the whole-lattice functions at every sampled
    site, including lattices two sites wide where the +mu and -mu neighbours coincide."""
    rng = np.random.default_rng(31)
    p = o.DWFParams(dims, 6, 1.8, 0.05, b, c)
    U = inputs.gauge_links(dims, 0.3, rng)
    n = int(np.prod(dims)) // 2
    x = rng.standard_normal((6, n, 4, 3)) + 1j * rng.standard_normal((6, n, 4, 3))
    sites = [0, 5, 17, n - 1]
    for dag, full in ((False, o.mpc(U, x, p)), (True, o.mpc_dag(U, x, p))):
        part = o.mpc_at_sites(U, x, p, sites, dag)
        assert np.abs(part - full[:, sites]).max() <= 1e-13 * np.abs(full).max()
