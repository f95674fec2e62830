"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle.

Element-by-element comparisons on identical seeded inputs:
  - FP64 storage: within 1e-12 max-abs per field (rho, u, T) after 1000 and
    2000 steps on the 129^2 Rayleigh-Benard case at Ra = 1e5;
  - every precision on tiny and ragged grids with random populations, every
    wall / periodic combination, one and several steps (edge and corner rules);
  - FP32 / FP16 / BF16 offset storage against FP64 within stated tolerances.
"""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

D2, D3 = 0, 1
FP64, FP32, FP16, BF16 = 0, 1, 2, 3


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    return tlbm


def _fields(sim):
    return {k: v.cpu().numpy() for k, v in sim.macros().items()}


def _maxerr(a, b, keys=("rho", "ux", "uy", "uz", "T")):
    return {k: float(np.abs(a[k] - b[k]).max()) for k in keys}


# ------------------------------------------------------------------ FP64 headline parity

@pytest.mark.parametrize("kw", [{}, {"streaming": 1}, {"walls": 1}], ids=["pull", "inplace", "side_heated"])
def test_fp64_2d_config1_1000_2000_steps(T, O, kw):
    """129^2, Ra = 1e5, Pr = 0.71, Ma = 0.1, RB walls, noise 1e-3, seed 1; the
    same with in-place streaming, and in the side-heated cavity."""
    g = T.Sim(129, 129, lattice=D2, Ra=1e5, Pr=0.71, Ma=0.1, precision=FP64, **kw)
    o = O.Sim(129, 129, lattice=D2, Ra=1e5, Pr=0.71, Ma=0.1, **{k: v for k, v in kw.items() if k != "streaming"})
    g.init(1, 1e-3)
    o.init(1, 1e-3)
    e0 = _maxerr(_fields(g), o.macros())
    assert max(e0.values()) < 1e-15, e0
    for target in (1000, 2000):
        g.step(target - o.time)
        o.step(target - o.time)
        e = _maxerr(_fields(g), o.macros())
        assert max(e.values()) < 1e-12, (target, e)
    assert abs(g.nusselt() - o.nusselt()) < 1e-10
    eg, mg = g.energy()
    eo, mo = o.energy()
    assert abs(mg - mo) / mo < 1e-12 and abs(eg - eo) < 1e-10 * eo
    fg, gg = g.get_populations()
    fo, go = o.get_populations()
    assert np.abs(fg - fo).max() < 1e-12 and np.abs(gg - go).max() < 1e-12


@pytest.mark.parametrize("kw", [{}, {"streaming": 1}], ids=["pull", "inplace"])
def test_fp64_3d_parity(T, O, kw):
    """D3Q19 + D3Q7 cube of 65^3 nodes, 500 steps (walls on every face), both
    streaming schemes."""
    n = 65
    g = T.Sim(n, n, n, lattice=D3, Ra=1e5, Pr=0.71, Ma=0.1, precision=FP64, **kw)
    o = O.Sim(n, n, n, lattice=D3, Ra=1e5, Pr=0.71, Ma=0.1)
    O.set_threads(8)
    g.init(3, 1e-3)
    o.init(3, 1e-3)
    g.step(500)
    o.step(500)
    e = _maxerr(_fields(g), o.macros())
    assert max(e.values()) < 1e-12, e
    assert abs(g.nusselt() - o.nusselt()) < 1e-10


# ------------------------------------------------------------------ edge cases, every precision

TOL1 = {FP64: 1e-14, FP32: 2e-6, FP16: 2e-3, BF16: 1.2e-2}

EDGE_CASES = [
    # lattice, (nx, ny, nz), walls, periodic mask
    (D2, (3, 3, 1), 0, 0), (D2, (4, 5, 1), 1, 0), (D2, (5, 4, 1), 0, 1), (D2, (7, 6, 1), 0, 2),
    (D2, (6, 3, 1), 1, 3), (D2, (37, 9, 1), 0, 0), (D2, (131, 5, 1), 0, 1), (D2, (257, 4, 1), 1, 0),
    (D3, (5, 4, 3), 0, 0), (D3, (3, 4, 5), 1, 0), (D3, (4, 3, 3), 0, 1), (D3, (3, 3, 4), 0, 6),
    (D3, (4, 3, 3), 1, 5), (D3, (35, 4, 3), 0, 0), (D3, (70, 3, 4), 0, 7),
]


# every compiled step variant: (vec, form) with form 1 = general MRT, 2 = TRT evaluation
VARIANTS = {
    (D2, FP32): [(4, 2), (2, 2), (1, 2), (4, 1)], (D2, FP16): [(8, 2), (4, 2), (2, 2), (8, 1)],
    (D2, BF16): [(8, 2), (4, 2), (2, 2), (8, 1)], (D2, FP64): [(2, 2), (1, 2), (2, 1)],
    (D3, FP32): [(4, 2), (2, 2), (1, 2), (2, 1)], (D3, FP16): [(4, 2), (2, 2), (1, 2), (4, 1)],
    (D3, BF16): [(4, 2), (2, 2), (1, 2), (4, 1)], (D3, FP64): [(1, 2), (2, 2), (1, 1)],
}
# software-pipelined variants: (vec, rows), two-relaxation-time form
ROW_VARIANTS = {
    (D2, FP32): [(4, 2), (4, 4)], (D2, FP16): [(4, 2), (4, 4), (8, 2), (8, 4)],
    (D2, BF16): [(4, 2), (4, 4), (8, 2), (8, 4)], (D2, FP64): [],
    (D3, FP32): [(1, 2), (1, 4)], (D3, FP16): [(1, 2), (1, 4)], (D3, BF16): [(1, 2), (1, 4)], (D3, FP64): [],
}


@pytest.mark.parametrize("prec", [FP64, FP32, FP16, BF16])
@pytest.mark.parametrize("lattice,shape,walls,pm", EDGE_CASES)
def test_one_step_random_populations(T, O, prec, lattice, shape, walls, pm):
    """Random populations set through the ABI; one and then two more steps must
    match the oracle started from the same values as the GPU stores them, for
    every compiled kernel variant (nodes per thread, MRT or TRT evaluation)."""
    nx, ny, nz = shape
    kw = dict(walls=walls, periodic_mask=pm)
    o = O.Sim(nx, ny, nz, lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1, **kw)
    qf, qg = (9, 5) if lattice == D2 else (19, 7)
    seed = 7 + 13 * lattice + 3 * walls + pm + 100 * prec + nx
    f = inputs.uniform_array(seed, (qf,) + o.shape, 0.02, 0.2)
    gg = inputs.uniform_array(seed + 1, (qg,) + o.shape, -0.1, 0.1)
    ref = None
    variants = [("reg", v, f, 1) for v, f in VARIANTS[(lattice, prec)]]
    variants += [("reg", v, 2, r) for v, r in ROW_VARIANTS[(lattice, prec)]]
    if prec != FP64:
        # shared-memory staged kernel: several tiles per row, 3 and 4 stages, and
        # whole rows
        A = 16 // (4 if prec == FP32 else 2)
        variants += [("staged", A, 3, 0), ("staged", 2 * A, 4, 0), ("staged", 0, 0, 0)]
    for kind, vec, form, rows in variants:
        g = T.Sim(nx, ny, nz, lattice=lattice, Ra=1e5, Pr=0.71, Ma=0.1, precision=prec, **kw)
        if kind == "staged":
            g.set_staged(vec, form)
            assert g.variant[0] == 0
        else:
            g.set_variant(vec, form, 0, 0, rows)
            assert g.variant[:2] == (vec, form) and g.variant[4] == rows
        g.set_populations(f, gg)
        f0, g0 = g.get_populations()  # as stored in the GPU precision
        if ref is None:
            o.set_populations(f0, g0)
            ref = []
            for n in (1, 2):
                o.step(n)
                ref.append(o.get_populations())
        for (fo, go), n in zip(ref, (1, 2)):
            g.step(n)
            fg, ggg = g.get_populations()
            ef = np.abs(fg - fo).max() / np.abs(fo).max()
            eg = np.abs(ggg - go).max() / np.abs(go).max()
            assert ef < TOL1[prec] * n and eg < TOL1[prec] * n, (vec, form, n, ef, eg)
        g.close()


def test_variants_agree_bitwise(T):
    """Nodes per thread, block shape and the shared-memory staged kernel change
    only how loads are issued: all TRT variants give bit-identical states."""
    for lattice, shape, prec in ((D2, (301, 45, 1), FP32), (D2, (301, 45, 1), FP16), (D3, (77, 21, 13), FP32),
                                 (D3, (77, 21, 13), BF16)):
        outs = []
        trt = [(v, 1) for v, f in VARIANTS[(lattice, prec)] if f == 2] + ROW_VARIANTS[(lattice, prec)]
        for vec, rows in trt:
            for bx, by in ((128, 1), (64, 2), (32, 4)):
                g = T.Sim(*shape, lattice=lattice, Ra=1e6, Pr=0.71, Ma=0.1, precision=prec)
                g.set_variant(vec, 2, bx, by, rows)
                g.init(11, 1e-3)
                g.step(20)
                outs.append(g.get_populations())
                g.close()
        for tw, ns in ((0, 0), (16, 3), (64, 4), (256, 0), (512 if lattice == D2 else 448, 2)):
            g = T.Sim(*shape, lattice=lattice, Ra=1e6, Pr=0.71, Ma=0.1, precision=prec)
            g.set_staged(tw, ns)
            g.init(11, 1e-3)
            g.step(20)
            outs.append(g.get_populations())
            g.close()
        for f, gg in outs[1:]:
            assert np.array_equal(f, outs[0][0]) and np.array_equal(gg, outs[0][1])


@pytest.mark.parametrize("prec", [FP64, FP32, FP16, BF16])
@pytest.mark.parametrize("lattice,shape", [(D2, (129, 65, 1)), (D3, (37, 20, 18))])
def test_init_matches_oracle(T, O, prec, lattice, shape):
    """Same counter-based noise on both sides: the initial temperature agrees
    to the storage precision, and exactly in FP64."""
    g = T.Sim(*shape, lattice=lattice, Ra=1e6, Pr=0.71, Ma=0.1, precision=prec)
    o = O.Sim(*shape, lattice=lattice, Ra=1e6, Pr=0.71, Ma=0.1)
    g.init(42, 1e-3)
    o.init(42, 1e-3)
    tg, to = _fields(g)["T"], o.macros()["T"]
    tol = {FP64: 2.5e-16, FP32: 1e-7, FP16: 1e-3, BF16: 8e-3}[prec]
    assert np.abs(tg - to).max() < tol


# ------------------------------------------------------------------ reduced precision vs FP64

@pytest.mark.parametrize("prec,tol_T,tol_u", [(FP32, 2e-5, 3e-5), (FP16, 4e-3, 6e-3), (BF16, 3e-2, 5e-2)])
def test_reduced_precision_fields_vs_oracle(T, O, prec, tol_T, tol_u):
    """129^2, Ra = 1e5, 400 steps: field error max|a - b| / max|b| (velocity
    components scaled by the largest velocity component).  Measured: FP32 T
    7.7e-6, u 1.2e-5; FP16 2.0e-3, 2.7e-3; BF16 1.5e-2, 2.5e-2 (16-bit storage
    rounding stochastically); the bounds are about twice those."""
    g = T.Sim(129, 129, lattice=D2, Ra=1e5, Pr=0.71, Ma=0.1, precision=prec)
    o = O.Sim(129, 129, lattice=D2, Ra=1e5, Pr=0.71, Ma=0.1)
    g.init(1, 1e-3)
    o.init(1, 1e-3)
    g.step(400)
    o.step(400)
    a, b = _fields(g), o.macros()
    umax = max(np.abs(b["ux"]).max(), np.abs(b["uy"]).max())
    rel = {"T": float(np.abs(a["T"] - b["T"]).max() / np.abs(b["T"]).max()),
           "ux": float(np.abs(a["ux"] - b["ux"]).max() / umax),
           "uy": float(np.abs(a["uy"] - b["uy"]).max() / umax)}
    print("field rel err", prec, rel)
    assert rel["T"] < tol_T and rel["ux"] < tol_u and rel["uy"] < tol_u, rel


# ------------------------------------------------------------------ bench-size sampled parity

@pytest.mark.parametrize("prec,tol", [(FP32, 3e-6), (FP16, 3e-3)])
def test_full_size_sampled_windows(T, O, prec, tol):
    """8193^2 at Ra = 1e8 in the benchmark's launch configuration: after a few
    steps, windows at a corner, a wall and the interior are read back; one
    oracle step on each window (with the full cell's parameters) must match the
    GPU's next state on the window's inner nodes."""
    n = 8193
    g = T.Sim(n, n, lattice=D2, Ra=1e8, Pr=0.71, Ma=0.1, precision=prec)
    d = g.derived()
    g.init(2, 1e-3)
    g.step(5)
    w = 24
    boxes = [(0, 0), (n - w, n - w), (4000, 0), (0, 5000), (n - w, 3000), (4090, 4090), (8000, n - w)]
    before = [g.get_window(x0, y0, 0, w, w) for x0, y0 in boxes]
    g.step(1)
    after = [g.get_window(x0, y0, 0, w, w) for x0, y0 in boxes]
    for (x0, y0), (f0, g0), (f1, g1) in zip(boxes, before, after):
        o = O.Sim(w, w, lattice=D2, Ra=1e8, Pr=0.71, Ma=0.1, nu=d["nu"], alpha=d["alpha"], gbeta=d["gbeta"])
        o.set_populations(f0, g0)
        o.step(1)
        fo, go = o.get_populations()
        # inner nodes: drop a side only where it is an artificial window edge
        xs = slice(0 if x0 == 0 else 1, w if x0 + w == n else w - 1)
        ys = slice(0 if y0 == 0 else 1, w if y0 + w == n else w - 1)
        ef = np.abs(f1[:, ys, xs] - fo[:, ys, xs]).max() / np.abs(fo).max()
        eg = np.abs(g1[:, ys, xs] - go[:, ys, xs]).max() / np.abs(go).max()
        assert ef < tol and eg < tol, ((x0, y0), ef, eg)
    div, step = g.status()
    assert not div and step == 6


@pytest.mark.parametrize("prec,tol", [(FP32, 3e-6), (FP16, 3e-3)])
def test_full_size_sampled_windows_3d(T, O, prec, tol):
    """385^3 at Ra = 1e7 in the benchmark's launch configuration: after a few
    steps, 12^3 windows at corners, on every face and in the interior are read
    back; one oracle step on each window (with the full cell's parameters) must
    match the GPU's next state on the window's inner nodes."""
    n, w = 385, 12
    g = T.Sim(n, n, n, lattice=D3, Ra=1e7, Pr=0.71, Ma=0.1, precision=prec)
    d = g.derived()
    g.init(3, 1e-3)
    g.step(5)
    e = n - w
    boxes = [(0, 0, 0), (e, e, e), (186, 0, 186), (0, 186, 186), (186, 186, 0), (186, 186, e), (e, 100, 250),
             (186, e, 40), (186, 186, 186), (0, e, 0)]
    before = [g.get_window(x0, y0, z0, w, w, w) for x0, y0, z0 in boxes]
    g.step(1)
    after = [g.get_window(x0, y0, z0, w, w, w) for x0, y0, z0 in boxes]
    for (x0, y0, z0), (f0, g0), (f1, g1) in zip(boxes, before, after):
        o = O.Sim(w, w, w, lattice=D3, Ra=1e7, Pr=0.71, Ma=0.1, nu=d["nu"], alpha=d["alpha"], gbeta=d["gbeta"])
        o.set_populations(f0, g0)
        o.step(1)
        fo, go = o.get_populations()
        # inner nodes: drop a side only where it is an artificial window edge
        sl = [slice(0 if c0 == 0 else 1, w if c0 + w == n else w - 1) for c0 in (x0, y0, z0)]
        ef = np.abs(f1[:, sl[2], sl[1], sl[0]] - fo[:, sl[2], sl[1], sl[0]]).max() / np.abs(fo).max()
        eg = np.abs(g1[:, sl[2], sl[1], sl[0]] - go[:, sl[2], sl[1], sl[0]]).max() / np.abs(go).max()
        assert ef < tol and eg < tol, ((x0, y0, z0), ef, eg)
    div, step = g.status()
    assert not div and step == 6
    g.close()


def test_mass_conserved_on_gpu(T):
    """FP64 storage: sum rho is constant to round-off over 1000 steps."""
    g = T.Sim(257, 129, lattice=D2, Ra=1e6, Pr=0.71, Ma=0.1, precision=FP64)
    g.init(5, 1e-3)
    m0 = g.energy()[1]
    g.step(1000)
    m1 = g.energy()[1]
    assert abs(m1 - m0) / m0 < 1e-13


def test_reductions_are_deterministic(T):
    g = T.Sim(513, 257, lattice=D2, Ra=1e7, Pr=0.71, Ma=0.1, precision=FP32)
    g.init(9, 1e-3)
    g.step(50)
    a = [g.nusselt() for _ in range(3)]
    assert a[0] == a[1] == a[2]


def test_divergence_is_reported(T):
    """A state with |u| > 0.5 is flagged by tlbm_status."""
    g = T.Sim(16, 16, lattice=D2, Ra=1e5, Pr=0.71, Ma=0.1, precision=FP64)
    f = np.zeros((9, 16, 16))
    gg = np.zeros((5, 16, 16))
    f[0] = 0.5
    f[1] = 0.6  # u_x = 0.6/1.1 > 0.5 at every node
    g.set_populations(f, gg)
    div, _ = g.status()
    assert div
    with pytest.raises(T.TlbmError) as ei:
        g.nusselt()
    assert ei.value.code == T.TLBM_ERR_DIVERGED
    assert g.nusselt(allow_diverged=True) == 1.0  # T = 0 everywhere
    g.init(1, 1e-3)
    assert not g.status()[0]
    g.nusselt()


@pytest.mark.parametrize("prec", [FP64, FP32, FP16, BF16])
def test_non_finite_state_is_reported(T, prec):
    """A NaN in the host buffer of tlbm_set_populations is found by the next
    reduction: tlbm_status flags it, tlbm_energy returns TLBM_ERR_DIVERGED, and
    a batch reports the one diverged instance."""
    g = T.Sim(24, 20, lattice=D2, Ra=1e5, Pr=0.71, Ma=0.1, precision=prec)
    g.init(2, 1e-3)
    f, gg = g.get_populations()
    f[4, 7, 9] = np.nan
    g.set_populations(f, gg)
    g.step(2)
    assert g.status()[0]
    with pytest.raises(T.TlbmError) as ei:
        g.energy()
    assert ei.value.code == T.TLBM_ERR_DIVERGED
    g.close()
    inst = [(17, 17, 1, 1e5, 0.71, 0.1, 1), (19, 17, 1, 1e5, 0.71, 0.1, 2)]
    b = T.Batch(inst, lattice=D2, precision=prec)
    b.init(1e-3)
    f, gg = b.get_populations(1)
    f[0, 3, 3] = np.inf
    T.tlbm_set_populations(b.instance(1), f, gg)
    b.step(1)
    assert b.status() == [False, True]
    with pytest.raises(T.TlbmError) as ei:
        b.nusselt()
    assert ei.value.code == T.TLBM_ERR_DIVERGED
    nu = b.nusselt(allow_diverged=True)
    assert np.isfinite(nu[0]) and not np.isfinite(nu[1])
    b.close()


def test_staged_at_bench_size(T):
    """The staged kernel on the 385^3 FP16 cube agrees bitwise with the register
    kernel after a few steps (whole-row tiles, the staged default in 3D)."""
    outs = []
    for staged in (False, True):
        g = T.Sim(385, 385, 385, lattice=D3, Ra=1e7, Pr=0.71, Ma=0.1, precision=FP16)
        if staged:
            g.set_staged()
        g.init(3, 1e-3)
        g.step(4)
        outs.append(g.get_window(180, 0, 0, 24, 24, 24))
        outs.append(g.get_window(361, 361, 361, 24, 24, 24))
        assert not g.status()[0]
        g.close()
    assert all(np.array_equal(a, b) for a, b in zip(outs[0] + outs[1], outs[2] + outs[3]))


def test_staged_default_configuration(T):
    """FP16/BF16 default to the staged kernel: in 2D 512-node tiles and the
    stage count that keeps at most six tiles in flight per SM, in 3D whole rows
    (up to 448 nodes) with 2 stages; tlbm_get_staged reports it, and the
    register kernels report zeros."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for prec in (FP16, BF16):
        g = T.Sim(1025, 257, lattice=D2, Ra=1e6, Pr=0.71, Ma=0.1, precision=prec)
        tw, ns, nb = g.staged
        assert tw == 512 and 2 <= ns <= 8 and nb % sms == 0 and (nb // sms) * ns <= 6, (tw, ns, nb)
        g.set_variant(4, 2, 32, 1, 1)
        assert g.staged == (0, 0, 0)
        g.close()
        g = T.Sim(385, 33, 33, lattice=D3, Ra=1e6, Pr=0.71, Ma=0.1, precision=prec)
        tw, ns, nb = g.staged
        assert tw == 392 and ns == 2 and nb % sms == 0, (tw, ns, nb)
        g.close()


def test_launch_count(T):
    g = T.Sim(64, 64, lattice=D2, Ra=1e5, Pr=0.71, Ma=0.1, precision=FP32)
    g.init(1, 0.0)
    c0 = g.launches
    g.step(10)
    assert g.launches - c0 == 10


def test_graph_replay_matches_plain_launches(T):
    """Steps replayed from the captured CUDA graph give the same bits as plain
    launches, for odd and even step counts and after a variant change."""
    for prec in (FP32, FP16):
        outs = []
        for gs in (0, 16, 6):
            g = T.Sim(131, 67, lattice=D2, Ra=1e6, Pr=0.71, Ma=0.1, precision=prec)
            T.tlbm_set_graph(g.h, gs)
            g.init(3, 1e-3)
            g.step(5)
            g.step(37)
            g.set_variant(2, 2, 0, 0, 1)
            g.step(20)
            assert g.launches == 1 + 62 and g.status()[1] == 62
            outs.append(g.get_populations())
            g.close()
        for f, gg in outs[1:]:
            assert np.array_equal(f, outs[0][0]) and np.array_equal(gg, outs[0][1])


def test_side_heated_cavity_is_centro_symmetric(T):
    """The side-heated cavity of §2.3 (hot left, cold right, adiabatic top and
    bottom): from the symmetric conductive start the state keeps the cavity's
    point symmetry, T(x, y) = -T(n-1-x, n-1-y) and u(x, y) = -u(n-1-x, n-1-y)."""
    n = 65
    g = T.Sim(n, n, lattice=D2, Ra=1e5, Pr=0.71, Ma=0.1, precision=FP64, walls=1)
    g.init(1, 0.0)
    g.step(6000)
    m = _fields(g)
    rot = lambda a: a[::-1, ::-1]
    assert np.abs(m["T"] + rot(m["T"])).max() < 1e-12
    assert np.abs(m["ux"] + rot(m["ux"])).max() < 1e-12 and np.abs(m["uy"] + rot(m["uy"])).max() < 1e-12
    assert np.abs(m["ux"]).max() > 1e-3  # a convective roll has formed
    assert g.nusselt() > 1.5
