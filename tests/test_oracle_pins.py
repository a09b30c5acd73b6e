"""Pins of the CPU oracle against what mechanics and mathematics fix.

None of these compares the oracle with itself: each check uses an independent
route (closed forms, a second derivation of k0 by exact 1-D integrals, other
library solvers, brute force, finite differences, beam theory).  The mutation
tests at the end plant plausible mistakes into copies of the oracle's element
matrix and check that the pins catch every one of them.
"""
import os

import numpy as np
import pytest

from oracle import fem

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


CONST = _golden("setup_constants.txt")
CLOSED = _golden("closed_forms.txt")
NU = CONST["nu"]


# ---------------------------------------------------------------- k0 pins
def k0_kronecker(h=1.0, nu=0.3):
    """Unit-E brick matrix from exact 1-D integrals (independent of quadrature).

    K[(a,p),(b,q)] = int lam dN_a/dx_p dN_b/dx_q + mu dN_a/dx_q dN_b/dx_p
                     + mu delta_pq grad N_a . grad N_b,
    and each 3-D integral is a product of 1-D integrals of the linear hat
    functions on [0, h]: int N N, int N' N, int N N', int N' N'.
    """
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    M = h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])          # int N_a N_b
    S = 1.0 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])        # int N_a' N_b'
    Dl = 0.5 * np.array([[-1.0, -1.0], [1.0, 1.0]])          # int N_a' N_b
    Dr = Dl.T                                                  # int N_a N_b'
    loc = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]

    def integral(a, b, da, db):
        # int (d/dx_da N_a or N_a) (d/dx_db N_b or N_b), da/db in {None, 0, 1, 2}
        val = 1.0
        for r in range(3):
            ia, ib = loc[a][r], loc[b][r]
            if da == r and db == r:
                val *= S[ia, ib]
            elif da == r:
                val *= Dl[ia, ib]
            elif db == r:
                val *= Dr[ia, ib]
            else:
                val *= M[ia, ib]
        return val

    K = np.zeros((24, 24))
    for a in range(8):
        for b in range(8):
            for p in range(3):
                for q in range(3):
                    v = lam * integral(a, b, p, q) + mu * integral(a, b, q, p)
                    if p == q:
                        v += mu * sum(integral(a, b, r, r) for r in range(3))
                    K[3 * a + p, 3 * b + q] = v
    return K


def linear_field(G, h=1.0):
    """Element DOFs of u(x) = G x for the unit-size brick scaled by h."""
    X = fem.LOCAL_NODES * h
    return np.concatenate([G @ X[a] for a in range(8)])


def pin_symmetric(k0):
    return np.abs(k0 - k0.T).max() < 1e-14


def pin_rigid_nullspace(k0):
    R = fem.rigid_body_modes()
    ev = np.linalg.eigvalsh(0.5 * (k0 + k0.T))
    return np.abs(k0 @ R).max() < 1e-13 and int((np.abs(ev) < 1e-12).sum()) == 6


def pin_constant_strain(k0, nu=NU):
    """u_e^T k0 u_e = V eps^T D eps for every constant-strain state (V = 1)."""
    lam, mu = CLOSED["lambda"], CLOSED["mu"]
    cases = [
        (np.diag([1.0, 0, 0]), lam + 2 * mu),                   # uniaxial strain
        (np.array([[0, 0.5, 0], [0.5, 0, 0], [0, 0, 0.0]]), mu),  # shear gamma_xy = 1
        (np.array([[0, 0, 0], [0, 0, 0.5], [0, 0.5, 0.0]]), mu),  # shear gamma_yz = 1
        (np.array([[0, 0, 0.5], [0, 0, 0], [0.5, 0, 0.0]]), mu),  # shear gamma_xz = 1
        (np.eye(3), 3 * (3 * lam + 2 * mu)),                     # dilatation: 9 K_bulk
        (np.diag([1.0, -1.0, 0]), 4 * mu),                        # pure shear in axes
    ]
    for G, energy in cases:
        ue = linear_field(G)
        if abs(ue @ k0 @ ue - energy) > 1e-13:
            return False
    return True


def pin_kronecker(k0):
    return np.abs(k0 - k0_kronecker(1.0, NU)).max() < 1e-14


def test_k0_symmetric_and_row_sums_zero():
    k0 = fem.element_stiffness(1.0, NU)
    assert pin_symmetric(k0)
    assert np.abs(k0.sum(axis=1)).max() < 1e-14      # translations are stress-free


def test_k0_nullspace_is_rigid_motions_rank18():
    k0 = fem.element_stiffness(1.0, NU)
    assert pin_rigid_nullspace(k0)
    assert np.linalg.matrix_rank(k0, tol=1e-10) == 18


def test_k0_matches_exact_one_dimensional_integrals():
    assert pin_kronecker(fem.element_stiffness(1.0, NU))


def test_k0_quadrature_is_exact():
    # B^T D B is at most quadratic per coordinate on a brick, so 2^3 Gauss points are exact
    k2 = fem.element_stiffness(1.0, NU, ngauss=2)
    k3 = fem.element_stiffness(1.0, NU, ngauss=3)
    assert np.abs(k2 - k3).max() < 1e-15


def test_k0_scales_linearly_with_h():
    k1 = fem.element_stiffness(1.0, NU)
    for h in (0.25, 2.0, 3.5):
        assert np.abs(fem.element_stiffness(h, NU) - h * k1).max() < 1e-13 * h


def test_k0_constant_strain_energies_and_diagonal():
    k0 = fem.element_stiffness(1.0, NU)
    assert pin_constant_strain(k0)
    assert np.allclose(np.diag(k0), CLOSED["k0_diag"], rtol=0, atol=1e-15)
    lam, mu = fem.lame(1.0, NU)
    assert abs(lam - CLOSED["lambda"]) < 1e-15 and abs(mu - CLOSED["mu"]) < 1e-15


# ---------------------------------------------------------------- mesh, BC, load
def test_load_totals_and_lines():
    g = fem.Grid(6, 4, 2)
    f = fem.load_vector(g, fem.LOAD_EDGE_XL_BOTTOM).reshape(-1, 3)
    assert abs(f[:, 2].sum() + 1.0) < 1e-15 and np.abs(f[:, :2]).max() == 0
    loaded = np.flatnonzero(f[:, 2])
    ijk = g.node_ijk()[loaded]
    assert (ijk[:, 0] == 6).all() and (ijk[:, 2] == 0).all() and len(loaded) == 5
    assert np.allclose(sorted(-f[loaded, 2]), [1 / 8, 1 / 8, 1 / 4, 1 / 4, 1 / 4])
    f = fem.load_vector(g, fem.LOAD_EDGE_X0_TOP).reshape(-1, 3)
    ijk = g.node_ijk()[np.flatnonzero(f[:, 2])]
    assert (ijk[:, 0] == 0).all() and (ijk[:, 2] == 2).all()
    f = fem.load_vector(fem.Grid(3, 2, 5, h=0.5), fem.LOAD_FACE_XL_TRACTION, 2.0).reshape(-1, 3)
    assert abs(f[:, 0].sum() - 2.0 * (2 * 0.5) * (5 * 0.5)) < 1e-14


def test_fixed_dofs_counts():
    g = fem.Grid(4, 2, 2)
    nn = 3 * 3
    assert fem.fixed_dofs(g, fem.BC_CANTILEVER).sum() == 3 * nn
    m = fem.fixed_dofs(g, fem.BC_MBB).reshape(-1, 3)
    assert m[:, 0].sum() == nn and m[:, 2].sum() == 3 and m[:, 1].sum() == 1
    with pytest.raises(ValueError):
        fem.fixed_dofs(fem.Grid(4, 3, 2), fem.BC_MBB)


# ---------------------------------------------------------------- assembly + solve
def test_patch_linear_field_interior_equilibrium():
    g = fem.Grid(4, 3, 3, h=0.7)
    k0 = fem.element_stiffness(g.h, NU)
    K = fem.assemble(g, np.ones(g.n_elem), k0)
    rng = np.random.default_rng(3)
    A, b = rng.normal(size=(3, 3)), rng.normal(size=3)
    X = g.node_ijk() * g.h
    u = (X @ A.T + b).reshape(-1)
    r = (K @ u).reshape(-1, 3)
    ijk = g.node_ijk()
    interior = ((ijk > 0) & (ijk < [g.nx, g.ny, g.nz])).all(axis=1)
    assert interior.sum() == 3 * 2 * 2
    assert np.abs(r[interior]).max() < 1e-13 * np.abs(u).max()


@pytest.mark.parametrize("shape,h", [((5, 3, 2), 0.5), ((3, 3, 3), 1.0)])
def test_uniaxial_tension_exact(shape, h):
    nx, ny, nz = shape
    t = 1.7
    P = fem.Problem(nx, ny, nz, fem.BC_ROLLER_BOX, fem.LOAD_FACE_XL_TRACTION,
                    np.ones(nx * ny * nz), Emin=0.0, h=h, load_magnitude=t)
    u = P.solve().reshape(-1, 3)
    X = P.grid.node_ijk() * h
    exact = np.stack([t * X[:, 0], -NU * t * X[:, 1], -NU * t * X[:, 2]], axis=1)
    assert np.abs(u - exact).max() < 1e-12
    V = nx * ny * nz * h ** 3
    assert abs(P.compliance(u.reshape(-1)) - t * t * V) < 1e-12 * t * t * V


def _random_problem(nx, ny, nz, bc, load, seed, lo=0.05):
    rho = np.random.default_rng(seed).uniform(lo, 1.0, nx * ny * nz)
    return fem.Problem(nx, ny, nz, bc, load, rho)


def test_direct_solves_agree_dense_banded_cg():
    P = _random_problem(6, 4, 4, fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM, 1)
    ud = fem.solve_direct(P.K, P.f, P.fixed, None)                  # dense Cholesky
    ub = fem.solve_direct(P.K, P.f, P.fixed, P.grid, dense_limit=10)  # banded Cholesky
    uc = fem.solve_cg(P.K, P.f, P.fixed, rtol=1e-14)
    n = np.linalg.norm(ud)
    assert np.linalg.norm(ub - ud) / n < 1e-12
    assert np.linalg.norm(uc - ud) / n < 1e-9
    assert P.rel_residual(ud) < 1e-12


def test_tiny_against_brute_force_dense_solve():
    # 1x1x1 cantilever: 4 free nodes, K_ff (12 x 12) built from k0 rows directly
    rho = np.array([0.6])
    P = fem.Problem(1, 1, 1, fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM, rho)
    k0 = fem.element_stiffness(1.0, NU)
    E = 1e-9 + 0.6 ** 3 * (1 - 1e-9)
    free_local = [1, 2, 5, 6]                     # local nodes with i = 1
    idx = [3 * a + c for a in free_local for c in range(3)]
    Kff = E * k0[np.ix_(idx, idx)]
    fl = np.zeros(12)
    fl[3 * 0 + 2] = -0.5                           # local node 1 = (1,0,0)
    fl[3 * 1 + 2] = -0.5                           # local node 2 = (1,1,0)
    ul = np.linalg.solve(Kff, fl)
    u = P.solve()
    g = P.grid
    nodes = [g.node(1, 0, 0), g.node(1, 1, 0), g.node(1, 0, 1), g.node(1, 1, 1)]
    got = np.concatenate([u[3 * n:3 * n + 3] for n in nodes])
    assert np.abs(got - ul).max() < 1e-10 * np.abs(ul).max()


def test_compliance_identity_and_energy():
    P = _random_problem(6, 4, 2, fem.BC_MBB, fem.LOAD_EDGE_X0_TOP, 2)
    u = P.solve()
    c1 = P.compliance(u)
    c2 = float(u @ (P.K @ u))
    c3 = fem.compliance_energy(P.grid, u, P.E, P.k0)
    assert c1 > 0
    assert abs(c1 - c2) < 1e-12 * c1 and abs(c1 - c3) < 1e-12 * c1


def test_operator_symmetry_on_random_vectors():
    P = _random_problem(5, 3, 3, fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM, 4)
    rng = np.random.default_rng(0)
    v, w = rng.normal(size=(2, P.grid.n_dof))
    assert abs(v @ (P.K @ w) - w @ (P.K @ v)) < 1e-12 * abs(v @ (P.K @ w))


def test_mbb_pin_position_changes_nothing_physical():
    P = _random_problem(6, 4, 2, fem.BC_MBB, fem.LOAD_EDGE_X0_TOP, 5)
    u1 = P.solve()
    # move the y pin from j = ny/2 to j = 0 on the same roller line
    g = P.grid
    fixed2 = P.fixed.copy()
    fixed2[3 * g.node(g.nx, g.ny // 2, 0) + 1] = False
    fixed2[3 * g.node(g.nx, 0, 0) + 1] = True
    u2 = fem.solve_direct(P.K, P.f, fixed2, None)
    assert abs(P.compliance(u1) - P.compliance(u2)) < 1e-11 * P.compliance(u1)
    e1 = fem.element_energies(g, u1, P.k0)
    e2 = fem.element_energies(g, u2, P.k0)
    assert np.abs(e1 - e2).max() < 1e-10 * e1.max()
    # the two solutions differ by a rigid y translation only
    d = (u2 - u1).reshape(-1, 3)
    assert np.abs(d[:, [0, 2]]).max() < 1e-9 * np.abs(u1).max()
    assert np.ptp(d[:, 1]) < 1e-9 * np.abs(u1).max()


def test_timoshenko_tip_deflection_converges_from_below():
    """Solid cantilever, L:b = 10, unit tip load: mean tip u_z approaches
    PL^3/(3EI) + PL/(kappa G A) monotonically from below as h -> 0."""
    ratios = []
    kappa = CLOSED["cowper_kappa"]
    for n in (4, 8, 12):
        L = 10 * n
        P = fem.Problem(L, n, n, fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM,
                        np.ones(L * n * n), Emin=0.0)
        u = P.solve()
        g = P.grid
        tip = [3 * g.node(L, j, k) + 2 for j in range(n + 1) for k in range(n + 1)]
        I = n ** 4 / 12.0
        G = 1.0 / (2 * (1 + NU))
        delta = L ** 3 / (3 * I) + L / (kappa * G * n * n)
        ratios.append(-u[tip].mean() / delta)
    assert ratios[0] < ratios[1] < ratios[2] < 1.0
    assert ratios[2] > 0.98 and ratios[0] > 0.9


# ---------------------------------------------------------------- sensitivities
@pytest.mark.parametrize("shape,bc,load", [((1, 1, 1), fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM),
                                           ((2, 1, 1), fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM),
                                           ((4, 2, 2), fem.BC_MBB, fem.LOAD_EDGE_X0_TOP)])
def test_sensitivity_central_differences(shape, bc, load):
    nx, ny, nz = shape
    rho = np.random.default_rng(7).uniform(0.2, 1.0, nx * ny * nz)
    P = fem.Problem(nx, ny, nz, bc, load, rho)
    dc = P.sensitivity(P.solve())
    delta = 1e-4
    for e in range(rho.size):
        cs = []
        for s in (+1, -1):
            r2 = rho.copy()
            r2[e] += s * delta
            Q = fem.Problem(nx, ny, nz, bc, load, r2)
            cs.append(Q.compliance(Q.solve()))
        fd = (cs[0] - cs[1]) / (2 * delta)
        assert abs(fd - dc[e]) <= 1e-6 * abs(dc[e]) + 1e-12, (e, fd, dc[e])


def test_sensitivity_uniform_scaling_law():
    """With Emin = 0, K(s rho) = s^p K(rho) so J(s) = J(1) s^-p and
    sum_e rho_e dJ/drho_e = -p J (Euler's theorem for a degree -p function)."""
    nx, ny, nz = 4, 2, 2
    for s in (0.3, 0.8):
        P = fem.Problem(nx, ny, nz, fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM,
                        np.full(nx * ny * nz, s), Emin=0.0)
        u = P.solve()
        J = P.compliance(u)
        dc = P.sensitivity(u)
        assert abs(dc.sum() * s + 3.0 * J) < 1e-11 * J
        Q = fem.Problem(nx, ny, nz, fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM,
                        np.ones(nx * ny * nz), Emin=0.0)
        assert abs(J - Q.compliance(Q.solve()) / s ** 3) < 1e-11 * J
    assert (dc < 0).all()


# ---------------------------------------------------------------- matrix-free pieces
def test_apply_at_nodes_matches_assembled():
    P = _random_problem(5, 4, 3, fem.BC_CANTILEVER, fem.LOAD_EDGE_XL_BOTTOM, 8)
    u = np.random.default_rng(1).normal(size=P.grid.n_dof)
    full = (P.K @ u).reshape(-1, 3)
    nodes = np.array([0, 7, 31, P.grid.n_nodes - 1, 55])
    got = fem.apply_at_nodes(P.grid, P.E, P.k0, u, nodes)
    assert np.abs(got - full[nodes]).max() < 1e-13 * np.abs(full).max()
    elems = np.array([0, 3, 17, P.grid.n_elem - 1])
    allv = fem.element_energies(P.grid, u, P.k0)
    assert np.allclose(fem.element_energies_at(P.grid, u, P.k0, elems), allv[elems], rtol=1e-13)


# ---------------------------------------------------------------- planted mistakes
def _mutants():
    k = fem.element_stiffness(1.0, NU)
    out = {}
    # engineering vs tensor shear strain mixed up: D shear = 2 mu
    D = fem.constitutive_matrix(1.0, NU)
    D2 = D.copy()
    D2[3, 3] = D2[4, 4] = D2[5, 5] = 2 * D[3, 3]
    out["shear_2mu"] = _k0_with(D2)
    # plane-stress-like lambda
    lam, mu = fem.lame(1.0, NU)
    D3 = D.copy()
    D3[:3, :3] = 2 * lam * mu / (lam + 2 * mu)
    for i in range(3):
        D3[i, i] = D3[0, 1] + 2 * mu
    out["wrong_lambda"] = _k0_with(D3)
    # two local nodes swapped (wrong local ordering)
    p = np.arange(24)
    p[[6, 7, 8, 9, 10, 11]] = [9, 10, 11, 6, 7, 8]
    out["swapped_nodes"] = k[np.ix_(p, p)]
    # one Gauss weight dropped
    out["dropped_point"] = k - _one_gauss_term()
    # transposed coupling block
    kt = k.copy()
    kt[0:3, 3:6] = k[0:3, 3:6].T
    out["transposed_block"] = kt
    return out


def _k0_with(D):
    pts, _ = np.polynomial.legendre.leggauss(2)
    K = np.zeros((24, 24))
    for a in pts:
        for b in pts:
            for c in pts:
                B = fem.strain_displacement(fem.shape_gradients(a, b, c) / 0.5)
                K += 0.125 * (B.T @ D @ B)
    return K


def _one_gauss_term():
    g = 1 / np.sqrt(3.0)
    B = fem.strain_displacement(fem.shape_gradients(g, g, g) / 0.5)
    return 0.125 * (B.T @ fem.constitutive_matrix(1.0, NU) @ B)


@pytest.mark.parametrize("name", ["shear_2mu", "wrong_lambda", "swapped_nodes", "dropped_point",
                                  "transposed_block"])
def test_pins_catch_planted_mistake(name):
    k = _mutants()[name]
    pins = [pin_symmetric(k), pin_rigid_nullspace(k), pin_constant_strain(k), pin_kronecker(k)]
    assert not all(pins), name


def test_paper_supports_and_loads():
    """Sec. 4.2/4.3 problems at the paper's 40x20x20: four 7x7-node corner
    patches (0.3 of 20 elements = 6 -> nodes 0..6 and 14..20), a disc and a
    half-disc load of total -1 that are symmetric about y = ny/2 (and z = nz/2)."""
    g = fem.Grid(40, 20, 20)
    m = fem.fixed_dofs(g, fem.BC_CORNERS).reshape(-1, 3)
    ijk = g.node_ijk()[m.any(axis=1)]
    assert m.sum() == 3 * 4 * 49 and (ijk[:, 0] == 0).all()
    assert set(ijk[:, 1]) == set(range(7)) | set(range(14, 21))
    m = fem.fixed_dofs(g, fem.BC_MBB_STRIP).reshape(-1, 3)
    assert m[:, 0].sum() == 21 * 21 and m[:, 2].sum() == 2 * 21 and m[:, 1].sum() == 1
    for load in (fem.LOAD_DISC_XL, fem.LOAD_HALFDISC_X0_TOP):
        f = fem.load_vector(g, load).reshape(-1, 3)
        assert abs(f[:, 2].sum() + 1.0) < 1e-14 and np.abs(f[:, :2]).max() == 0
        F = f[:, 2].reshape(21, 21, 41)  # [k][j][i]
        assert np.allclose(F, F[:, ::-1, :])  # mirror in y about ny/2
        if load == fem.LOAD_DISC_XL:
            assert np.allclose(F, F[::-1, :, :]) and np.count_nonzero(F[:, :, :40]) == 0
        else:
            assert np.count_nonzero(F[:20]) == 0 and np.count_nonzero(F[20, :, 4:]) == 0
