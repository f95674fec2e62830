"""Pins of the oracle's time stepping against what physics and mathematics fix:
conservation, exact steady states, closed-form decay rates, linear-algebra
eigenvalues of the one-mode update, mirror symmetry and convection onset.
"""
import numpy as np
import pytest

D2, D3 = 0, 1


def _mirror_index(e, axis):
    q = len(e)
    out = np.zeros(q, dtype=int)
    for i in range(q):
        m = e[i].copy()
        m[axis] = -m[axis]
        out[i] = [j for j in range(q) if (e[j] == m).all()][0]
    return out


# ------------------------------------------------------------------ conservation

@pytest.mark.parametrize("lattice,shape", [(D2, (65, 33, 1)), (D3, (9, 8, 10))])
def test_mass_conserved_to_roundoff(O, lattice, shape):
    """Bounce-back and the Guo source add no mass: sum rho is constant."""
    nx, ny, nz = shape
    s = O.Sim(nx, ny, nz, lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1)
    s.init(1, 1e-3)
    m0 = s.energy()[1]
    s.step(400)
    m1 = s.energy()[1]
    assert abs(m1 - m0) / m0 < 1e-13
    assert s.energy()[0] > 0.0


@pytest.mark.parametrize("lattice,shape,pm", [(D2, (33, 17, 1), 2), (D3, (7, 6, 8), 4)])
def test_temperature_conserved_with_adiabatic_walls(O, lattice, shape, pm):
    """With the isothermal axis made periodic every wall is adiabatic, so the
    total temperature sum T is conserved (bounce-back of g, §2.2)."""
    nx, ny, nz = shape
    s = O.Sim(nx, ny, nz, lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1, periodic_mask=pm)
    s.init(3, 1e-2)
    T0 = s.macros()["T"].sum()
    s.step(300)
    T1 = s.macros()["T"].sum()
    assert abs(T1 - T0) < 1e-12


# ------------------------------------------------------------------ conduction

@pytest.mark.parametrize("lattice,shape,walls", [
    (D2, (8, 32, 1), 0), (D2, (24, 9, 1), 1), (D3, (5, 6, 16), 0), (D3, (12, 5, 4), 1)])
def test_pure_conduction_is_exact(O, lattice, shape, walls):
    """Buoyancy off: the linear conductive profile between the isothermal walls
    is reproduced to round-off by anti-bounce-back, u stays 0 and Nu = 1."""
    nx, ny, nz = shape
    s = O.Sim(nx, ny, nz, lattice=lattice, Ra=1e4, Pr=0.71, Ma=0.1, walls=walls, gbeta=0.0)
    s.init(1, 0.0)
    s.step(3000)
    m = s.macros()
    L = (ny if lattice == D2 else nz) if walls == 0 else nx
    c = (np.arange(L) + 0.5) / L
    lin = 0.5 - c
    if walls == 0:
        expect = lin[:, None] if lattice == D2 else lin[:, None, None]
    else:
        expect = lin[None, :] if lattice == D2 else lin[None, None, :]
    assert np.abs(m["T"] - expect).max() < 1e-15
    for k in ("ux", "uy", "uz"):
        assert np.abs(m[k]).max() == 0.0
    assert abs(s.nusselt() - 1.0) < 1e-14


@pytest.mark.slow
def test_subcritical_conduction_converges_second_order(O):
    """Ra = 1000 (below onset), buoyancy on, 1D layer (periodic x): the steady
    state is the conductive one up to the scheme's O(h^2) error in the
    hydrostatic balance; the deviation falls ~4x per grid doubling."""
    errs = []
    for ny in (16, 32, 64):
        s = O.Sim(4, ny, Ra=1000.0, Pr=0.71, Ma=0.1, periodic_mask=1)
        s.init(1, 0.0)
        s.step(int(8000 * (ny / 32) ** 2))
        m = s.macros()
        lin = 0.5 - (np.arange(ny) + 0.5) / ny
        errs.append((np.abs(m["uy"]).max(), np.abs(m["T"] - lin[:, None]).max(), abs(s.nusselt() - 1)))
    errs = np.array(errs)
    for k in range(2):
        r1, r2 = errs[0, k] / errs[1, k], errs[1, k] / errs[2, k]
        assert 3.0 < r1 < 8.0 and 3.0 < r2 < 8.0, errs
    assert errs[1, 0] < 1e-5 and errs[1, 2] < 1e-4


def test_noisy_subcritical_start_relaxes(O):
    """From the seeded noisy start (amplitude 1e-3) at Ra = 1000 the state
    relaxes to the steady state of the noise-free start.  What is left, a few
    1e-9, is a staggered (row-alternating) velocity mode that the scheme does not
    damp, the kind of spurious invariant that the paper's odd grid sizes (§2.3)
    are meant to weaken."""
    a = O.Sim(5, 17, Ra=1000.0, Pr=0.71, Ma=0.1, periodic_mask=1)
    b = O.Sim(5, 17, Ra=1000.0, Pr=0.71, Ma=0.1, periodic_mask=1)
    a.init(1, 0.0)
    b.init(5, 1e-3)
    a.step(12000)
    b.step(12000)
    assert np.abs(a.macros()["T"] - b.macros()["T"]).max() < 1e-8


# ------------------------------------------------------------------ Poiseuille

@pytest.mark.parametrize("lattice,ny", [(D2, 9), (D2, 16), (D3, 11)])
def test_poiseuille_exact_at_magic_parameter(O, lattice, ny):
    """Periodic along the flow, walls half-way outside the first/last node,
    body force a_x, buoyancy off: u_x(y) = a/(2 nu) (y+1/2)(N - 1/2 - y) holds to
    round-off with the 3/16 magic combination of rates."""
    a, nu = 1e-5, 0.1
    if lattice == D2:
        s = O.Sim(4, ny, Ra=1e5, Pr=0.71, Ma=0.1, periodic_mask=1, gbeta=0.0, nu=nu,
                  body_force=[a, 0, 0])
    else:
        s = O.Sim(4, 3, ny, lattice=D3, Ra=1e5, Pr=0.71, Ma=0.1, periodic_mask=3, gbeta=0.0,
                  nu=nu, body_force=[a, 0, 0])
    s.init(0, 0.0)
    s.step(int(14 * ny * ny / (nu * np.pi ** 2) * 2.3))
    m = s.macros()
    c = np.arange(ny) + 0.5
    exact = a / (2 * nu) * c * (ny - c)
    ux = m["ux"][:, 0] if lattice == D2 else m["ux"][:, 0, 0]
    assert np.abs(ux - exact).max() / exact.max() < 1e-10
    assert np.abs(m["uy"]).max() < 1e-14


def test_poiseuille_slip_error_away_from_magic(O):
    """With the odd rate moved off the magic value the half-way wall is no
    longer exact: a visible O(1/N^2) slip error appears and shrinks with N."""
    errs = []
    for ny in (9, 17):
        s = O.Sim(4, ny, Ra=1e5, Pr=0.71, Ma=0.1, periodic_mask=1, gbeta=0.0, nu=0.1,
                  body_force=[1e-5, 0, 0], s_q=1.0, s_e=1.0)
        s.init(0, 0.0)
        s.step(int(14 * ny * ny / (0.1 * np.pi ** 2) * 2.3))
        c = np.arange(ny) + 0.5
        exact = 1e-5 / 0.2 * c * (ny - c)
        errs.append(np.abs(s.macros()["ux"][:, 0] - exact).max() / exact.max())
    assert errs[0] > 1e-4
    assert 2.5 < errs[0] / errs[1] < 5.5


def test_conserved_rates_have_no_effect(O):
    """The Guo form makes the momentum update independent of s_j (and the mass
    update of s_rho)."""
    outs = []
    for sj in (1.0, 0.7, 1.6):
        s = O.Sim(17, 13, Ra=1e5, Pr=0.71, Ma=0.1, s_j=sj, s_rho=sj)
        s.init(2, 1e-3)
        s.step(200)
        outs.append(s.get_populations()[0])
    assert np.abs(outs[0] - outs[1]).max() < 1e-14
    assert np.abs(outs[0] - outs[2]).max() < 1e-14


# ------------------------------------------------------------------ decay rates

def _phase(e, k):
    return np.exp(-1j * (e @ k))


def _thermal_update_matrix(O, lattice, a_T, Q, k):
    """One-mode linear update of g at rest: G(k) = diag(exp(-i k.e)) (I - N^-1 Q (N - E))."""
    e, _, _, N, Ni = O.velocity_set(1 if lattice == D2 else 3)
    q = len(N)
    c = np.zeros(q)
    c[0] = 1.0
    c[3 if lattice == D2 else 4] = a_T
    E = np.outer(c, np.ones(q))
    C = np.eye(q) - Ni @ np.diag(Q) @ (N - E)
    return np.diag(_phase(e, k)) @ C


def _flow_update_matrix(O, lattice, S, k):
    """One-mode linear update of f about rest: f_eq linearised as w_i (rho + 3 e_i.j)."""
    e, w, _, M, Mi = O.velocity_set(0 if lattice == D2 else 2)
    q = len(M)
    J = np.array([[w[i] * (1.0 + 3.0 * e[i] @ e[j]) for j in range(q)] for i in range(q)])
    C = np.eye(q) - Mi @ np.diag(S) @ (M - M @ J)
    return np.diag(_phase(e, k)) @ C


@pytest.mark.parametrize("lattice", [D2, D3])
def test_thermal_mode_decay(O, lattice):
    """T = A sin(k x), fluid at rest, periodic: the amplitude ratio per step is
    the dominant eigenvalue of the one-mode update to round-off, and equals
    exp(-alpha k^2) up to O(k^4)."""
    nx = 64
    alpha = 0.05
    if lattice == D2:
        s = O.Sim(nx, 3, Ra=1e5, Pr=0.71, Ma=0.1, periodic_mask=3, gbeta=0.0, alpha=alpha)
    else:
        s = O.Sim(nx, 3, 3, lattice=D3, Ra=1e5, Pr=0.71, Ma=0.1, periodic_mask=7, gbeta=0.0,
                  alpha=alpha)
    d = s.derived()
    f, g = s.get_populations()
    e, w, *_ = O.velocity_set(0 if lattice == D2 else 2)
    f[:] = w.reshape((-1,) + (1,) * (f.ndim - 1))
    T = 1e-3 * np.sin(2 * np.pi * np.arange(nx) / nx)
    g1 = O.thermal_geq(lattice, d["a_T"], 1.0, [0, 0, 0])
    g[:] = g1.reshape((-1,) + (1,) * (g.ndim - 1)) * T
    s.set_populations(f, g)
    s.step(150)
    t0 = s.macros()["T"].reshape(-1, nx)[0, nx // 4]
    s.step(1)
    t1 = s.macros()["T"].reshape(-1, nx)[0, nx // 4]
    ratio = t1 / t0
    k = np.array([2 * np.pi / nx, 0.0, 0.0])
    lam = np.linalg.eigvals(_thermal_update_matrix(O, lattice, d["a_T"], d["Q"], k))
    dom = lam[np.argmax(lam.real)]
    assert abs(dom.imag) < 1e-12
    assert abs(ratio - dom.real) < 1e-12
    assert abs(ratio - np.exp(-alpha * k[0] ** 2)) / (1 - ratio) < 2e-3


@pytest.mark.parametrize("lattice", [D2, D3])
def test_shear_wave_decay(O, lattice):
    """u_x = A sin(k y), periodic, buoyancy off: the decay ratio is an
    eigenvalue of the linearised one-mode update and equals exp(-nu k^2) up to O(k^4)."""
    ny, nu, A = 48, 0.08, 1e-6
    if lattice == D2:
        s = O.Sim(3, ny, Ra=1e5, Pr=0.71, Ma=0.1, periodic_mask=3, gbeta=0.0, nu=nu)
    else:
        s = O.Sim(3, ny, 3, lattice=D3, Ra=1e5, Pr=0.71, Ma=0.1, periodic_mask=7, gbeta=0.0, nu=nu)
    d = s.derived()
    f, g = s.get_populations()
    e, w, _, M, Mi = O.velocity_set(0 if lattice == D2 else 2)
    g[:] = 0.0
    for y in range(ny):
        u = [A * np.sin(2 * np.pi * y / ny), 0.0, 0.0]
        fe = Mi @ O.flow_meq(lattice, 1.0, u)
        if lattice == D2:
            f[:, y, :] = fe[:, None]
        else:
            f[:, :, y, :] = fe[:, None, None]
    s.set_populations(f, g)
    s.step(300)
    ux = s.macros()["ux"]
    sel = (lambda a: a[ny // 4, 0]) if lattice == D2 else (lambda a: a[0, ny // 4, 0])
    u0 = sel(ux)
    s.step(1)
    u1 = sel(s.macros()["ux"])
    ratio = u1 / u0
    k = np.array([0.0, 2 * np.pi / ny, 0.0])
    lam = np.linalg.eigvals(_flow_update_matrix(O, lattice, d["S"], k))
    real = lam[np.abs(lam.imag) < 1e-12].real
    assert np.min(np.abs(real - ratio)) < 1e-9
    assert abs(ratio - np.exp(-nu * k[1] ** 2)) / (1 - ratio) < 5e-3


# ------------------------------------------------------------------ symmetry

@pytest.mark.parametrize("lattice,shape", [(D2, (33, 24, 1)), (D3, (9, 7, 10))])
def test_mirror_symmetry_preserved(O, lattice, shape):
    """A start that is mirror-symmetric in x stays so (to round-off growth):
    f_i(x) = f_mirror(i)(nx-1-x), g likewise."""
    nx, ny, nz = shape
    s = O.Sim(nx, ny, nz, lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1)
    s.init(9, 0.0)
    d = s.derived()
    f, g = s.get_populations()
    rng = np.random.default_rng(9)
    noise = rng.uniform(-1e-3, 1e-3, size=g.shape[1:])
    noise = 0.5 * (noise + noise[..., ::-1])
    g1 = O.thermal_geq(lattice, d["a_T"], 1.0, [0, 0, 0])
    g = g + g1.reshape((-1,) + (1,) * noise.ndim) * noise
    s.set_populations(f, g)
    s.step(500)
    f, g = s.get_populations()
    ef = O.velocity_set(0 if lattice == D2 else 2)[0]
    eg = O.velocity_set(1 if lattice == D2 else 3)[0]
    mf, mg = _mirror_index(ef, 0), _mirror_index(eg, 0)
    assert np.abs(f - f[mf][..., ::-1]).max() < 1e-13
    assert np.abs(g - g[mg][..., ::-1]).max() < 1e-13
    assert np.abs(s.macros()["ux"]).max() > 1e-9  # the start does drive a flow


# ------------------------------------------------------------------ onset

@pytest.mark.slow
def test_convection_onset_near_1708(O):
    """Rigid-rigid layer, periodic x with Nx = 2 Ny (k = pi/H, next to the
    critical wavenumber 3.117/H): the growth rate of a small perturbation of the
    conductive state changes sign within 2% of the textbook Ra_c = 1707.76."""
    ny = 32
    nx = 2 * ny
    rates = []
    ras = (1600.0, 1700.0, 1800.0)
    for Ra in ras:
        base = O.Sim(nx, ny, Ra=Ra, Pr=0.71, Ma=0.1, periodic_mask=1)
        base.init(0, 0.0)
        base.step(6000)
        d = base.derived()
        f, g = base.get_populations()
        x = np.arange(nx)
        y = np.arange(ny) + 0.5
        dT = 1e-6 * np.sin(np.pi * y / ny)[:, None] * np.cos(2 * np.pi * x / nx)[None, :]
        g1 = O.thermal_geq(0, d["a_T"], 1.0, [0, 0, 0])
        pert = O.Sim(nx, ny, Ra=Ra, Pr=0.71, Ma=0.1, periodic_mask=1)
        pert.set_populations(f, g + g1[:, None, None] * dT[None])
        ts, amps = [], []
        for k in range(7):
            n = 2000 if k == 0 else 1000
            base.step(n)
            pert.step(n)
            if k:
                mb, mp = base.macros(), pert.macros()
                amps.append(np.sqrt(((mp["ux"] - mb["ux"]) ** 2 + (mp["uy"] - mb["uy"]) ** 2).sum()))
                ts.append(pert.time)
        rates.append(np.polyfit(ts, np.log(amps), 1)[0])
    assert rates[0] < 0 < rates[2]
    p = np.polyfit(ras, rates, 1)
    ra_c = -p[1] / p[0]
    assert abs(ra_c / 1707.76 - 1) < 0.02, ra_c


# ------------------------------------------------------------------ coupling and diagnostics

@pytest.mark.parametrize("lattice,shape", [(D2, (9, 12, 1)), (D3, (7, 6, 9))])
def test_buoyancy_enters_the_velocity_along_gravity(O, lattice, shape):
    """Fluid at rest (sum e f = 0): u = F/(2 rho) with F = rho g beta T along +y
    in 2D and +z in 3D (§2.2), so u = g beta T / 2 on that axis, 0 elsewhere."""
    nx, ny, nz = shape
    s = O.Sim(nx, ny, nz, lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1)
    s.init(4, 1e-2)
    d = s.derived()
    m = s.macros()
    up, others = ("uy", ("ux", "uz")) if lattice == D2 else ("uz", ("ux", "uy"))
    assert np.abs(m[up] - 0.5 * d["gbeta"] * m["T"]).max() < 1e-18
    for k in others:
        assert np.abs(m[k]).max() == 0.0


@pytest.mark.parametrize("walls", [0, 1])
def test_nusselt_of_a_uniform_flow(O, walls):
    """Nu = 1 + L <u_h T> / (alpha dT) evaluated on a uniform state: u_h = U0
    and T = T0 everywhere give Nu = 1 + L U0 T0 / alpha (the definition used for
    the Nusselt number, L the extent along the heat-flux axis)."""
    nx, ny = 12, 9
    s = O.Sim(nx, ny, Ra=1e5, Pr=0.71, Ma=0.1, walls=walls, gbeta=0.0)
    d = s.derived()
    U0, T0 = 0.02, 0.3
    u = [U0, 0.0, 0.0] if walls == 1 else [0.0, U0, 0.0]
    e, w, _, M, Mi = O.velocity_set(0)
    feq = Mi @ O.flow_meq(0, 1.0, u)
    geq = O.thermal_geq(0, d["a_T"], T0, u)
    f = np.broadcast_to(feq[:, None, None], (9, ny, nx)).copy()
    g = np.broadcast_to(geq[:, None, None], (5, ny, nx)).copy()
    s.set_populations(f, g)
    L = nx if walls == 1 else ny
    assert abs(s.nusselt() - (1.0 + L * U0 * T0 / d["alpha"])) < 1e-12
