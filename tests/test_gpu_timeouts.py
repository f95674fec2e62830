"""The bounded waits of the staged kernel (for its copies) and of the
persistent batched kernel (at its grid barrier) give up and report
TLBM_ERR_TIMEOUT when their time limit runs out.  The tests set the limit to 0,
so that the first wait that has not already completed gives up: nothing faults
or hangs, the error stays reported until the state is initialised again, and the
handle then steps exactly as a fresh one."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    return tlbm


def test_staged_copy_wait_times_out_and_recovers(T):
    kw = dict(lattice=0, Ra=1e6, Pr=0.71, Ma=0.1, precision=T.TLBM_FP16_OFFSET)
    s = T.Sim(1025, 257, **kw)
    assert s.variant[0] == 0  # the staged kernel is the default for 2D FP16
    s.set_wait_limit(0)
    s.init(5, 1e-3)
    s.step(6)
    with pytest.raises(T.TlbmError) as ei:
        s.nusselt()
    assert ei.value.code == T.TLBM_ERR_TIMEOUT
    s.step(20)  # graph-captured steps; the error stays reported
    with pytest.raises(T.TlbmError) as ei:
        s.energy()
    assert ei.value.code == T.TLBM_ERR_TIMEOUT
    s.set_wait_limit(0.2)
    s.init(5, 1e-3)
    s.step(30)
    ref = T.Sim(1025, 257, **kw)
    ref.set_variant(4, 2, 32, 1, 1)  # the register kernel, bitwise the same arithmetic
    ref.init(5, 1e-3)
    ref.step(30)
    (fa, ga), (fb, gb) = s.get_populations(), ref.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert s.nusselt() == ref.nusselt()
    s.close()
    ref.close()


def test_persistent_barrier_wait_times_out_and_recovers(T):
    inst = []
    for N, Ra, Pr, seed in inputs.ensemble_draws(11, 4, sizes=(65, 97), log_ra=(5.0, 6.0)):
        inst.append((N, N, 1, Ra, Pr, 0.1, seed))
    b = T.Batch(inst, lattice=0, precision=T.TLBM_FP32)
    ref = T.Batch(inst, lattice=0, precision=T.TLBM_FP32)
    v = ref.variant
    b.set_variant(v[0], v[1], v[2], v[3], 0)
    b.set_persistent(8)
    b.set_wait_limit(0)
    b.init(1e-3)
    b.step(16)
    with pytest.raises(T.TlbmError) as ei:
        b.status()
    assert ei.value.code == T.TLBM_ERR_TIMEOUT
    b.step(8)  # a later launch resets the barrier, not the reported timeout
    with pytest.raises(T.TlbmError) as ei:
        b.status()
    assert ei.value.code == T.TLBM_ERR_TIMEOUT
    b.set_wait_limit(0.5)
    b.init(1e-3)
    b.step(16)
    assert b.status() == [False] * 4
    ref.init(1e-3)
    ref.step(16)
    for k in range(4):
        (fa, ga), (fb, gb) = b.get_populations(k), ref.get_populations(k)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb), k
    b.close()
    ref.close()
