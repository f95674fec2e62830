"""Pins of the oracle's tables and single-node algebra (no time stepping).

Each check compares the oracle with something fixed outside it: values the
paper prints (tests/golden/), textbook closed forms, or exact identities.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------- velocity sets

def test_d2q9_ordering_matches_halo_sets(O):
    """§3.1: f_{2,5,6}, g_2 move up (+y); f_{4,7,8}, g_4 move down."""
    e9 = O.velocity_set(0)[0]
    e5 = O.velocity_set(1)[0]
    sets = {ln[0]: [int(v) for v in ln[1:]] for ln in _golden_lines("halo_directions.txt")}
    assert sorted(np.nonzero(e9[:, 1] == 1)[0].tolist()) == sets["f_up"]
    assert sorted(np.nonzero(e9[:, 1] == -1)[0].tolist()) == sets["f_down"]
    assert np.nonzero(e5[:, 1] == 1)[0].tolist() == sets["g_up"]
    assert np.nonzero(e5[:, 1] == -1)[0].tolist() == sets["g_down"]


@pytest.mark.parametrize("which,q", [(0, 9), (1, 5), (2, 19), (3, 7)])
def test_velocity_sets_are_symmetric(O, which, q):
    e, w, opp, M, Mi = O.velocity_set(which)
    assert e.shape == (q, 3)
    assert len({tuple(v) for v in e}) == q
    for i in range(q):
        assert (e[opp[i]] == -e[i]).all()
    assert (np.abs(e) <= 1).all()


@pytest.mark.parametrize("which", [0, 2])
def test_flow_weights_isotropy(O, which):
    """Textbook lattice isotropy: sum w = 1, sum w e e = I/3, 4th moment = (dd+dd+dd)/9."""
    e, w, *_ = O.velocity_set(which)
    assert abs(w.sum() - 1.0) < 1e-15
    D = 2 if which == 0 else 3
    second = np.einsum("i,ia,ib->ab", w, e, e)[:D, :D]
    assert np.allclose(second, np.eye(D) / 3.0, atol=1e-15)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)[:D, :D, :D, :D]
    I = np.eye(D)
    expect = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
              + np.einsum("ad,bc->abcd", I, I)) / 9.0
    assert np.allclose(fourth, expect, atol=1e-15)
    odd = np.einsum("i,ia,ib,ic->abc", w, e, e, e)
    assert np.abs(odd).max() < 1e-15


@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_moment_matrix_orthogonal_and_inverse(O, which):
    """Rows of M (N) are mutually orthogonal integer vectors, and the oracle's
    Gauss-Jordan inverse satisfies M^-1 M = I."""
    e, w, opp, M, Mi = O.velocity_set(which)
    assert np.array_equal(M, np.round(M))
    G = M @ M.T
    assert np.array_equal(G, np.diag(np.diag(G)))
    assert np.abs(Mi @ M - np.eye(len(M))).max() < 1e-15
    # exact inverse M^T diag(1/|row|^2), computed in rationals
    q = len(M)
    for i in range(q):
        for k in range(q):
            exact = Fraction(int(M[k, i])) / Fraction(int(G[k, k]))
            assert abs(Mi[i, k] - float(exact)) <= 2e-16


def test_d2q9_rows_lallemand_luo(O):
    """Lallemand & Luo (2000) D2Q9 basis in the §3.1 ordering."""
    M = O.velocity_set(0)[3]
    expect = np.array([
        [1, 1, 1, 1, 1, 1, 1, 1, 1],
        [-4, -1, -1, -1, -1, 2, 2, 2, 2],
        [4, -2, -2, -2, -2, 1, 1, 1, 1],
        [0, 1, 0, -1, 0, 1, -1, -1, 1],
        [0, -2, 0, 2, 0, 1, -1, -1, 1],
        [0, 0, 1, 0, -1, 1, 1, -1, -1],
        [0, 0, -2, 0, 2, 1, 1, -1, -1],
        [0, 1, -1, 1, -1, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 1, -1, 1, -1],
    ], dtype=float)
    assert np.array_equal(M, expect)


# ---------------------------------------------------------------- forcing, Eq. (6)

def _eval(expr, u, F):
    env = dict(u=u[0], v=u[1], w=u[2], Fx=F[0], Fy=F[1], Fz=F[2],
               uF=u[0] * F[0] + u[1] * F[1] + u[2] * F[2])
    return eval(expr, {"__builtins__": {}}, env)


@pytest.mark.parametrize("lattice,tag,q", [(0, "D2Q9", 9), (1, "D3Q19", 19)])
def test_forcing_moments_match_printed_eq6(O, lattice, tag, q):
    """M * Ftilde (Guo forcing) equals the vector printed in Eq. (6a)/(6b)."""
    rows = {int(ln[1]): " ".join(ln[2:]) for ln in _golden_lines("forcing_moments_eq6.txt") if ln[0] == tag}
    assert sorted(rows) == list(range(q))
    r = inputs.rng(11)
    for trial in range(20):
        u = r.uniform(-0.1, 0.1, 3)
        F = r.uniform(-1e-3, 1e-3, 3)
        if lattice == 0:
            u[2] = 0.0
            F[2] = 0.0
        got = O.forcing_moments(lattice, u, F)
        want = np.array([_eval(rows[k], u, F) for k in range(q)])
        assert np.abs(got - want).max() <= 1e-17 + 1e-13 * np.abs(want).max()


def test_printed_d2q9_last_entry_is_a_typo(O):
    """With F = (0, Fy) the printed u Fx + v Fy differs from M*Ftilde; the read
    u Fy + v Fx matches (the reading recorded in the golden file)."""
    printed = [" ".join(ln[2:]) for ln in _golden_lines("forcing_moments_eq6.txt") if ln[0] == "D2Q9_printed"][0]
    u = np.array([0.03, -0.02, 0.0])
    F = np.array([0.0, 1e-4, 0.0])
    got = O.forcing_moments(0, u, F)[8]
    assert abs(got - _eval(printed, u, F)) > 1e-7
    assert abs(got - _eval("u*Fy + v*Fx", u, F)) < 1e-18


# ---------------------------------------------------------------- equilibria

def test_d2q9_meq_closed_form(O):
    """Lallemand & Luo (2000): m_eq = [rho, -2rho + 3rho|u|^2, rho - 3rho|u|^2,
    rho u, -rho u, rho v, -rho v, rho(u^2 - v^2), rho u v]."""
    r = inputs.rng(3)
    for _ in range(10):
        rho = r.uniform(0.9, 1.1)
        u, v = r.uniform(-0.1, 0.1, 2)
        uu = u * u + v * v
        want = [rho, -2 * rho + 3 * rho * uu, rho - 3 * rho * uu, rho * u, -rho * u,
                rho * v, -rho * v, rho * (u * u - v * v), rho * u * v]
        got = O.flow_meq(0, rho, [u, v, 0.0])
        assert np.abs(got - want).max() < 1e-15


def test_d3q19_meq_closed_form(O):
    """d'Humieres et al. (2002): e_eq = -11 rho + 19 rho|u|^2,
    eps_eq = 3 rho - 11/2 rho|u|^2, q_eq = -2/3 j, 3p_xx = rho(2u^2 - v^2 - w^2),
    pi_xx = -1/2 * 3p_xx, p_ww = rho(v^2 - w^2), pi_ww = -1/2 p_ww, p_ab = rho u_a u_b, m = 0."""
    r = inputs.rng(4)
    for _ in range(10):
        rho = r.uniform(0.9, 1.1)
        u, v, w = r.uniform(-0.1, 0.1, 3)
        uu = u * u + v * v + w * w
        pxx = rho * (2 * u * u - v * v - w * w)
        pww = rho * (v * v - w * w)
        want = [rho, -11 * rho + 19 * rho * uu, 3 * rho - 5.5 * rho * uu,
                rho * u, -2 / 3 * rho * u, rho * v, -2 / 3 * rho * v, rho * w, -2 / 3 * rho * w,
                pxx, -0.5 * pxx, pww, -0.5 * pww, rho * u * v, rho * v * w, rho * u * w, 0, 0, 0]
        got = O.flow_meq(1, rho, [u, v, w])
        assert np.abs(got - want).max() < 4e-16 * np.abs(want).max()


@pytest.mark.parametrize("lattice,tag", [(0, "D2Q5"), (1, "D3Q7")])
def test_antibounceback_omega_is_twice_moving_weight(O, lattice, tag):
    """§2.2: with omega from the printed formula, anti-bounce-back maps the
    wall-temperature equilibrium onto itself: -g_eq,i(Tw) + omega Tw = g_eq,ibar(Tw)."""
    (_, num, den), = [ln for ln in _golden_lines("anti_bounce_back_omega.txt") if ln[0] == tag]
    e, _, opp, _, _ = O.velocity_set(1 if lattice == 0 else 3)
    for a_T in (-2 / 3, -0.75, -0.5, 0.0, 1.0):
        omega = (float(num) + a_T) / float(den)
        for Tw in (0.5, -0.5, 0.123):
            geq = O.thermal_geq(lattice, a_T, Tw, [0.0, 0.0, 0.0])
            for i in range(1, len(geq)):
                assert abs(-geq[i] + omega * Tw - geq[opp[i]]) < 1e-16
            # c_sT^2 = sum_i geq_i e_ix^2 / T = omega
            assert abs(np.dot(geq, e[:, 0] ** 2) / Tw - omega) < 1e-15


@pytest.mark.parametrize("lattice", [0, 1])
def test_thermal_equilibrium_moments(O, lattice):
    """sum g_eq = T and sum e g_eq = u T (the temperature and its advective flux)."""
    e = O.velocity_set(1 if lattice == 0 else 3)[0]
    r = inputs.rng(5)
    for _ in range(10):
        T = r.uniform(-0.5, 0.5)
        u = r.uniform(-0.1, 0.1, 3)
        if lattice == 0:
            u[2] = 0
        geq = O.thermal_geq(lattice, -2 / 3 if lattice == 0 else -0.75, T, u)
        assert abs(geq.sum() - T) < 4e-16
        assert np.abs(e.T @ geq - u * T).max() < 4e-17


def test_default_thermal_weights(O):
    """a_T = -2/3 gives D2Q5 weights 1/3, 1/6; a_T = -3/4 gives D3Q7 weights 1/4, 1/8."""
    g5 = O.thermal_geq(0, -2 / 3, 1.0, [0, 0, 0])
    assert np.allclose(g5, [1 / 3] + [1 / 6] * 4, atol=1e-16)
    g7 = O.thermal_geq(1, -0.75, 1.0, [0, 0, 0])
    assert np.allclose(g7, [1 / 4] + [1 / 8] * 6, atol=1e-16)


# ---------------------------------------------------------------- parameter mapping

def test_parameter_mapping_free_fall_units(O):
    """Eqs. (2)-(4): nu/(U H) = sqrt(Pr/Ra), alpha/(U H) = 1/sqrt(Pr Ra),
    g beta dT H = U^2, Ra = g beta dT H^3/(nu alpha), Pr = nu/alpha."""
    s = O.Sim(129, 129, Ra=1e5, Pr=0.71, Ma=0.1)
    d = s.derived()
    assert abs(d["U"] - 0.1 / np.sqrt(3.0)) < 1e-16
    assert d["H"] == 129
    assert abs(d["gbeta"] * 1.0 * d["H"] ** 3 / (d["nu"] * d["alpha"]) / 1e5 - 1) < 1e-13
    assert abs(d["nu"] / d["alpha"] / 0.71 - 1) < 1e-13
    assert abs(d["gbeta"] * d["H"] / d["U"] ** 2 - 1) < 1e-13
    # 3D: H is the z extent
    s3 = O.Sim(9, 11, 13, lattice=O.D3Q19_D3Q7, Ra=1e7, Pr=0.71, Ma=0.1)
    assert s3.derived()["H"] == 13


def test_relaxation_rates_defaults(O):
    """Shear rate from nu = (1/s_nu - 1/2)/3; odd rates at the 3/16 magic
    parameter; thermal flux rate from alpha = c_sT^2 (1/q_j - 1/2)."""
    s = O.Sim(64, 64, Ra=1e6, Pr=0.71, Ma=0.1)
    d = s.derived()
    S, Q = d["S"], d["Q"]
    snu = S[7]
    assert abs((1 / snu - 0.5) / 3 - d["nu"]) < 1e-16
    assert S[1] == snu and S[2] == snu and S[8] == snu
    lam = (1 / snu - 0.5) * (1 / S[4] - 0.5)
    assert abs(lam - 3 / 16) < 1e-15
    assert abs(d["omega"] * (1 / Q[1] - 0.5) - d["alpha"]) < 1e-16
    assert abs((1 / Q[1] - 0.5) * (1 / Q[3] - 0.5) - 0.25) < 1e-15


@pytest.mark.parametrize("args", [
    dict(nx=2, ny=10), dict(nx=10, ny=2), dict(nx=10, ny=10, Ra=0.0), dict(nx=10, ny=10, Pr=-1.0),
    dict(nx=10, ny=10, Ma=0.0), dict(nx=10, ny=10, nu=1e-8),
])
def test_oracle_rejects_invalid(O, args):
    kw = dict(Ra=1e5, Pr=0.71, Ma=0.1)
    kw.update(args)
    nx, ny = kw.pop("nx"), kw.pop("ny")
    with pytest.raises(ValueError):
        O.Sim(nx, ny, **kw)


def test_init_random_numbers(O):
    """splitmix64-based uniform: in [0,1), a multiple of 2^-53, reproducible."""
    vals = [O.uniform(7, i) for i in range(1000)]
    assert all(0.0 <= v < 1.0 for v in vals)
    assert all(float(v * 2 ** 53).is_integer() for v in vals)
    assert abs(np.mean(vals) - 0.5) < 0.05
    assert O.uniform(7, 3) == vals[3]
    assert O.uniform(8, 3) != vals[3]
