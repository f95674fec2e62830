"""Reduced-precision storage against FP64, stated per result.

Laminar (129^2, Ra = 2e4: convection sets in after ~40 free-fall times from the
noisy conductive state and is a steady single roll by 100; compared after 120): field
error max|a - b| / max|b| of T and of the velocity (components scaled by the
largest FP64 velocity component), and the Nusselt number.

Chaotic (257^2, Ra = 1e7 and 1e8, Pr = 0.71): time-averaged Nusselt number over
60 free-fall times.  A single chaotic run's 60-free-fall-time average scatters
by several percent (the volume-averaged Nu fluctuates by ~40 % and the roll
settles into different configurations), so the comparison is paired: FP64
develops 8 states from 8 seeds over 20 free-fall times, and every storage
precision continues each of the same 8 states.

The FP64 comparator is the GPU FP64 path; each test first checks it against the
CPU oracle over the opening 2000 steps of its own case, to 1e-12.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

D2 = 0
FP64, FP32, FP16, BF16 = 0, 1, 2, 3
NAMES = {FP64: "fp64", FP32: "fp32", FP16: "fp16", BF16: "bf16"}
U = 0.1 / math.sqrt(3.0)  # free-fall velocity in lattice units (Ma = 0.1)


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


def _check_fp64_against_oracle(T, O, n, Ra, seed):
    """The GPU FP64 path equals the oracle over 2000 steps of the case (1e-12)."""
    O.set_threads(8)
    g = T.Sim(n, n, lattice=D2, Ra=Ra, Pr=0.71, Ma=0.1, precision=FP64)
    o = O.Sim(n, n, lattice=D2, Ra=Ra, Pr=0.71, Ma=0.1)
    g.init(seed, 1e-3)
    o.init(seed, 1e-3)
    g.step(2000)
    o.step(2000)
    a, b = _fields(g), o.macros()
    err = max(float(np.abs(a[k] - b[k]).max()) for k in ("rho", "ux", "uy", "T"))
    g.close()
    assert err < 1e-12, err


# (T, u, Nu) relative errors allowed at the laminar steady state, about twice
# the measured ones (FP32 1.7e-4, 3.7e-4, 1.5e-4; FP16 5.3e-3, 5.4e-3, 5.7e-3;
# BF16 1.9e-2, 2.5e-2, 2.2e-2)
LAMINAR_TOL = {FP32: (4e-4, 8e-4, 3e-4), FP16: (1.1e-2, 1.1e-2, 1.2e-2), BF16: (4e-2, 5e-2, 4.5e-2)}


def _field_errors(a, b, umax):
    """Relative field errors of a against b, or against b's mirror image in x
    when that is closer: the cell is mirror-symmetric and the noise picks the
    sense of the roll."""
    def errs(bT, bux, buy):
        eT = float(np.abs(a["T"] - bT).max() / np.abs(bT).max())
        eu = float(max(np.abs(a["ux"] - bux).max(), np.abs(a["uy"] - buy).max()) / umax)
        return eT, eu
    direct = errs(b["T"], b["ux"], b["uy"])
    mirror = errs(b["T"][:, ::-1], -b["ux"][:, ::-1], b["uy"][:, ::-1])
    return min(direct, mirror, key=lambda e: e[0] + e[1])


def test_laminar_steady_state_fields(T, O):
    n, Ra, seed = 129, 2e4, 1
    _check_fp64_against_oracle(T, O, n, Ra, seed)
    steps = int(120 * n / U)
    last = int(4 * n / U)
    out = {}
    for prec in (FP64, FP32, FP16, BF16):
        g = T.Sim(n, n, lattice=D2, Ra=Ra, Pr=0.71, Ma=0.1, precision=prec)
        g.init(seed, 1e-3)
        g.step(steps - last)
        nu_before = g.nusselt()
        # Nu averaged over the last 4 free-fall times (16-bit storage keeps a
        # small jitter: its stochastic rounding never settles exactly)
        nus = []
        for _ in range(16):
            g.step(last // 16)
            nus.append(g.nusselt())
        g.step(last - 16 * (last // 16))
        out[prec] = (_fields(g), float(np.mean(nus)))
        if prec == FP64:
            # steady: Nu unchanged over the last 4 free-fall times
            print(f"laminar fp64: Nu {nu_before:.9f} -> {nus[-1]:.9f}")
            assert abs(nus[-1] - nu_before) < 1e-6 * nu_before
        g.close()
    b, nu_ref = out[FP64]
    umax = max(np.abs(b["ux"]).max(), np.abs(b["uy"]).max())
    assert nu_ref > 1.5  # a convecting roll, not the conductive state
    for prec in (FP32, FP16, BF16):
        a, nu = out[prec]
        eT, eu = _field_errors(a, b, umax)
        enu = abs(nu - nu_ref) / nu_ref
        print(f"laminar {NAMES[prec]}: T {eT:.3e} u {eu:.3e} Nu {nu:.6f} vs {nu_ref:.6f} ({enu:.3e})")
        tT, tu, tnu = LAMINAR_TOL[prec]
        assert eT < tT and eu < tu and enu < tnu, (prec, eT, eu, enu)


def _paired_nusselt(T, n, Ra, nseed, t_dev, t_rec):
    """Per precision, per developed state: time-averaged Nu over t_rec free-fall
    times (sampled 16 times per free-fall time)."""
    tf = n / U
    every = int(tf / 16)
    inst = [(n, n, 1, Ra, 0.71, 0.1, 100 + k) for k in range(nseed)]
    b = T.Batch(inst, lattice=D2, precision=FP64)
    b.init(1e-3)
    b.step(int(t_dev * tf))
    states = [b.get_populations(k) for k in range(nseed)]
    b.close()
    means = {}
    for prec in (FP64, FP32, FP16, BF16):
        b = T.Batch(inst, lattice=D2, precision=prec)
        for k, (f, g) in enumerate(states):
            T.tlbm_set_populations(b.instance(k), np.ascontiguousarray(f), np.ascontiguousarray(g))
        series = []
        for _ in range(int(t_rec * 16)):
            b.step(every)
            series.append(b.nusselt())
        assert not any(b.status())
        b.close()
        means[prec] = np.array(series).mean(0)
    return means


@pytest.mark.parametrize("Ra", [1e7, 1e8])
def test_chaotic_time_averaged_nusselt(T, O, Ra):
    n = 257
    _check_fp64_against_oracle(T, O, n, Ra, 100)
    means = _paired_nusselt(T, n, Ra, 8, 20.0, 60.0)
    ref = means[FP64]
    for prec in (FP32, FP16, BF16):
        d = (means[prec] - ref) / ref
        med = float(np.median(d))
        print(f"Ra {Ra:g} {NAMES[prec]}: ensemble {means[prec].mean():.4f} vs {ref.mean():.4f} "
              f"({means[prec].mean() / ref.mean() - 1:+.4f}); paired median {med:+.4f}; per state {np.round(d, 4)}")
        # every state keeps convecting (round-to-nearest 16-bit storage froze
        # into steady rolls 40 % below FP64)
        assert means[prec].min() > 0.75 * ref.min()
        assert abs(med) < CHAOTIC_TOL[prec], (prec, med)


# |paired median relative difference| of the time-averaged Nu allowed per
# storage precision: FP32 meets the 1 % criterion; the 16-bit formats, with
# stochastic rounding, carry a systematic error of a few percent (measured: FP16
# -5.0 % at Ra 1e7, +2.3 % at 1e8; BF16 +6.1 %, -0.5 %)
CHAOTIC_TOL = {FP32: 0.01, FP16: 0.06, BF16: 0.08}
