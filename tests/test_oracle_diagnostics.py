"""Pins of the oracle's diagnostics and of its initial-state random numbers
against values fixed outside the oracle:

- mass sum rho and kinetic energy 1/2 sum rho |u|^2 of a state built in the test
  from given per-node rho, u, T (the macroscopic moments of §2.2: rho = sum f,
  u = (sum e f + F/2) / rho with the Boussinesq force F = rho g beta T g_hat);
- the splitmix64 output function behind the initial-state noise, against the
  published output sequence of the generator for seed 0.
"""
import os

import numpy as np
import pytest

D2, D3 = 0, 1
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# textbook lattice weights by |e|^2 (D2Q9: 4/9, 1/9, 1/36; D3Q19: 1/3, 1/18, 1/36)
WEIGHTS = {D2: {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}, D3: {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}}
GOLDEN_RATIO_64 = 0x9E3779B97F4A7C15


def _state_with_macros(O, lattice, shape, rho, u, T, gbeta):
    """Populations whose moments are the given rho, u, T: f = f_eq(rho, u - F/(2 rho))
    (the second-order equilibrium has sum f = rho and sum e f = rho times its
    velocity exactly on these lattices), g_0 = T and the other g zero."""
    e = O.velocity_set(0 if lattice == D2 else 2)[0].astype(np.float64)
    w = np.array([WEIGHTS[lattice][int(v @ v)] for v in e])
    gax = 1 if lattice == D2 else 2
    F = np.zeros(u.shape)
    F[..., gax] = rho * gbeta * T
    v = u - F / (2.0 * rho[..., None])
    eu = np.einsum("qa,...a->q...", e, v)
    vv = (v * v).sum(-1)
    f = w.reshape((-1,) + (1,) * rho.ndim) * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * vv)
    qg = 5 if lattice == D2 else 7
    g = np.zeros((qg,) + rho.shape)
    g[0] = T
    return f, g


@pytest.mark.parametrize("lattice,shape", [(D2, (23, 17, 1)), (D3, (7, 6, 5))])
def test_energy_and_mass_of_a_given_state(O, lattice, shape):
    nx, ny, nz = shape
    s = O.Sim(nx, ny, nz, lattice=lattice, Ra=1e6, Pr=0.71, Ma=0.1)
    gbeta = s.derived()["gbeta"]
    assert gbeta > 0
    r = np.random.default_rng(11 + lattice)
    sh = s.shape
    rho = r.uniform(0.9, 1.1, sh)
    u = r.uniform(-0.05, 0.05, sh + (3,))
    if lattice == D2:
        u[..., 2] = 0.0
    T = r.uniform(-0.5, 0.5, sh)
    f, g = _state_with_macros(O, lattice, shape, rho, u, T, gbeta)
    s.set_populations(f, g)
    m = s.macros()
    assert np.abs(m["rho"] - rho).max() < 1e-14
    assert np.abs(m["ux"] - u[..., 0]).max() < 1e-14
    assert np.abs(m["uy"] - u[..., 1]).max() < 1e-14
    assert np.abs(m["uz"] - u[..., 2]).max() < 1e-14
    ekin, mass = s.energy()
    ekin_ref = 0.5 * (rho * (u * u).sum(-1)).sum()
    assert abs(mass - rho.sum()) <= 1e-13 * rho.sum()
    assert abs(ekin - ekin_ref) <= 1e-12 * ekin_ref


@pytest.mark.parametrize("lattice", [D2, D3])
def test_energy_and_mass_of_a_uniform_flow(O, lattice):
    """Closed form: a uniform state rho0, U0 gives mass rho0 N and kinetic
    energy rho0 |U0|^2 N / 2 (buoyancy off so that F = 0)."""
    shape = (9, 8, 1) if lattice == D2 else (5, 4, 6)
    s = O.Sim(*shape, lattice=lattice, Ra=1e6, Pr=0.71, Ma=0.1, gbeta=0.0)
    rho0, U0 = 1.05, np.array([0.03, -0.02, 0.0 if lattice == D2 else 0.01])
    sh = s.shape
    f, g = _state_with_macros(O, lattice, shape, np.full(sh, rho0), np.broadcast_to(U0, sh + (3,)).copy(),
                              np.zeros(sh), 0.0)
    s.set_populations(f, g)
    ekin, mass = s.energy()
    N = s.N
    assert abs(mass - rho0 * N) <= 1e-13 * rho0 * N
    assert abs(ekin - 0.5 * rho0 * float(U0 @ U0) * N) <= 1e-12 * ekin


def _published_splitmix64():
    out = {}
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as fh:
        for ln in fh:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                k, v = ln.split()
                out[int(k)] = int(v)
    return out


def test_uniform_uses_splitmix64_published_outputs(O):
    """tlbmo_uniform(seed, idx) = top 53 bits of splitmix64(seed ^ splitmix64(idx)) x 2^-53.
    With the published outputs z_k = splitmix64((k - 1) * golden) the inner and
    outer arguments can be steered onto known points of the sequence."""
    z = _published_splitmix64()
    M = (1 << 64) - 1
    top = lambda v: (v >> 11) * 2.0 ** -53
    # inner splitmix64(0) = z_1; seed = z_1 ^ golden makes the outer argument golden -> z_2
    assert O.uniform(z[1] ^ GOLDEN_RATIO_64, 0) == top(z[2])
    # inner splitmix64(golden) = z_2; seed = z_2 makes the outer argument 0 -> z_1
    assert O.uniform(z[2], GOLDEN_RATIO_64) == top(z[1])
    # inner splitmix64(2 golden) = z_3; outer argument 3 golden -> z_4
    assert O.uniform(z[3] ^ ((3 * GOLDEN_RATIO_64) & M), (2 * GOLDEN_RATIO_64) & M) == top(z[4])
    # and the draws lie in [0, 1)
    vals = [O.uniform(7, i) for i in range(1000)]
    assert min(vals) >= 0.0 and max(vals) < 1.0
