"""tlbm_reduce_noalloc: the diagnostic sums for callers that cannot allocate
device memory, checked through the C ABI against the handle-based entry points
(tlbm_nusselt, tlbm_energy, tlbm_status) on two calls in a row.

Collected last on purpose: it runs the library's static scratch path after
every other GPU test has used the handle-based one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    return tlbm


def _check_against_handle_path(T, sim, sums):
    nu_ref = sim.nusselt()
    ekin_ref, mass_ref = sim.energy()
    div_ref, _ = sim.status()
    d = sim.derived()
    ax = 0 if sim.params.walls == T.TLBM_SIDE_HEATED else (1 if sim.lattice == 0 else 2)
    L = (sim.nx, sim.ny, sim.nz)[ax]
    nu = 1.0 + L * (sums[0] / sim.N) / (d["alpha"] * 1.0)
    assert abs(nu - nu_ref) <= 1e-12 * abs(nu_ref)
    assert abs(sums[1] - ekin_ref) <= 1e-12 * abs(ekin_ref)
    assert abs(sums[2] - mass_ref) <= 1e-12 * abs(mass_ref)
    assert (sums[4] != 0.0 or not (sums[3] <= 0.25)) == div_ref


@pytest.mark.parametrize("lattice,shape,prec", [(0, (1031, 517, 1), 1), (0, (129, 129, 1), 0), (1, (97, 65, 49), 2),
                                                 (1, (33, 33, 33), 3)])
def test_noalloc_matches_handle_reductions_twice(T, lattice, shape, prec):
    sim = T.Sim(*shape, lattice=lattice, Ra=1e7, Pr=0.71, Ma=0.1, precision=prec)
    sim.init(4, 1e-3)
    sim.step(30)
    first = T.tlbm_reduce_noalloc(sim.h)
    _check_against_handle_path(T, sim, first)
    second = T.tlbm_reduce_noalloc(sim.h)
    assert first == second  # same state, same fixed summation order
    sim.step(7)
    third = T.tlbm_reduce_noalloc(sim.h)
    _check_against_handle_path(T, sim, third)
    assert third != first


def test_noalloc_with_explicit_state_pointer(T):
    """A state passed by device address (buffer 0 of a bound block after an even
    number of steps) to a handle that has no memory bound."""
    shape = (257, 129, 1)
    sim = T.Sim(*shape, lattice=0, Ra=1e6, Pr=0.71, Ma=0.1, precision=1)
    sim.init(8, 1e-3)
    sim.step(12)
    ref = T.tlbm_reduce_noalloc(sim.h)
    h = T.tlbm_create(*shape, 0, 1e6, 0.71, 0.1, 1)
    try:
        a = T.tlbm_reduce_noalloc(h, sim.mem.data_ptr())
        b = T.tlbm_reduce_noalloc(h, sim.mem.data_ptr())
    finally:
        T.tlbm_destroy(h)
    assert a == ref and b == ref


def test_noalloc_rejects_oversize_and_unbound(T):
    big = T.tlbm_create(11600, 11600, 1, 0, 1e8, 0.71, 0.1, 2)
    try:
        sim = T.Sim(64, 64, lattice=0, Ra=1e6, Pr=0.71, Ma=0.1, precision=2)
        with pytest.raises(T.TlbmError) as ei:
            T.tlbm_reduce_noalloc(big, sim.mem.data_ptr())
        assert ei.value.code == T.TLBM_ERR_ARG
        assert "static scratch" in T.tlbm_last_error(big)
        with pytest.raises(T.TlbmError) as ei:
            T.tlbm_reduce_noalloc(big)
        assert ei.value.code == T.TLBM_ERR_ARG
    finally:
        T.tlbm_destroy(big)
    small = T.tlbm_create(64, 64, 1, 0, 1e6, 0.71, 0.1, 1)
    try:
        with pytest.raises(T.TlbmError) as ei:
            T.tlbm_reduce_noalloc(small)
        assert ei.value.code == T.TLBM_ERR_UNBOUND
    finally:
        T.tlbm_destroy(small)


def test_noalloc_flags_divergence(T):
    sim = T.Sim(16, 16, lattice=0, Ra=1e5, Pr=0.71, Ma=0.1, precision=0)
    f = np.zeros((9, 16, 16))
    g = np.zeros((5, 16, 16))
    f[0] = 0.5
    f[1] = 0.6
    sim.set_populations(f, g)
    s = T.tlbm_reduce_noalloc(sim.h)
    assert s[3] > 0.25 and sim.status()[0]


def test_noalloc_in_place_state_order(T):
    """In-place streaming keeps the state in natural order after an even number
    of steps and in swapped order after an odd number; a state passed by pointer
    is read in the order of the handle's own current state."""
    shape = (131, 67, 1)
    sim = T.Sim(*shape, lattice=0, Ra=1e6, Pr=0.71, Ma=0.1, precision=1, streaming=T.TLBM_STREAM_INPLACE)
    sim.init(5, 1e-3)
    sim.step(11)  # odd: swapped order
    own = T.tlbm_reduce_noalloc(sim.h, sim.mem.data_ptr())
    _check_against_handle_path(T, sim, own)
    assert own == T.tlbm_reduce_noalloc(sim.h)
    sim.step(1)  # even: natural order, as a fresh handle reads it
    ref = T.tlbm_reduce_noalloc(sim.h)
    _check_against_handle_path(T, sim, ref)
    params = T.tlbm_default_params(streaming=T.TLBM_STREAM_INPLACE)
    h = T.tlbm_create(*shape, 0, 1e6, 0.71, 0.1, 1, params)
    try:
        a = T.tlbm_reduce_noalloc(h, sim.mem.data_ptr())
        b = T.tlbm_reduce_noalloc(h, sim.mem.data_ptr())
    finally:
        T.tlbm_destroy(h)
    assert a == ref and b == ref


def test_noalloc_call_allocates_no_device_memory(T):
    """After the first call on the device (which looks up the static array's
    address), further calls leave the device's free memory and torch's
    allocator untouched."""
    import torch

    sim = T.Sim(513, 257, lattice=0, Ra=1e7, Pr=0.71, Ma=0.1, precision=2)
    sim.init(6, 1e-3)
    sim.step(4)
    first = T.tlbm_reduce_noalloc(sim.h)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    again = [T.tlbm_reduce_noalloc(sim.h) for _ in range(3)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    assert stats1.get("allocation.all.allocated", 0) == stats0.get("allocation.all.allocated", 0)
    assert all(a == first for a in again)
