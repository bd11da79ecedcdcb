"""Failure paths through the C ABI, injected on the host or by a wait limit: nothing here faults,
traps or hangs the GPU.

- invalid input: NaN integrals, a non-Hermitian two-electron tensor, NaN or mislabelled MPS
  tensors, truncated or corrupt checkpoint files -> SPMPS_ERR_BAD_INPUT, no device work;
- an iteration cap of one Davidson iteration -> SPMPS_ERR_NOT_CONVERGED with the sweep finished;
- a target spin no state of the sector has (P = 0) -> SPMPS_ERR_SINGULAR_METRIC;
- the bounded mbarrier wait of the tensor-core inference kernel given one poll -> it gives up
  (SPMPS_ERR_TIMEOUT), still waits for its MMAs in flight with the default limit, frees its
  tensor memory, and the context stays usable.
"""
import numpy as np
import pytest

from paper_1703_04789_gb300 import inputs
from tests.gpu_util import require_gpu

BAD_INPUT, NOT_CONVERGED, SINGULAR_METRIC, TIMEOUT = 1, 2, 3, 5


def _spmps(*a, **kw):
    from paper_1703_04789_gb300 import Spmps
    return Spmps(*a, **kw)


@pytest.mark.gpu
def test_invalid_integrals_are_rejected():
    require_gpu()
    from paper_1703_04789_gb300 import SpmpsError
    K = 4
    h1, h2, _ = inputs.synthetic_active_space(K, 3)
    dev = _spmps(K, 4, 0, 0, 3, 8)
    bad = h1.copy()
    bad[1, 2] = np.nan
    with pytest.raises(SpmpsError) as ei:
        dev.set_hamiltonian(bad, h2)
    assert ei.value.status == BAD_INPUT
    nh = h2.copy()
    nh[0, 1, 2, 3] += 0.1  # breaks (pq|rs) = (qp|sr)
    with pytest.raises(SpmpsError) as ei:
        dev.set_hamiltonian(h1, nh)
    assert ei.value.status == BAD_INPUT
    nan2 = h2.copy()
    nan2[1, 1, 2, 2] = np.nan
    with pytest.raises(SpmpsError) as ei:
        dev.set_hamiltonian(h1, nan2)
    assert ei.value.status == BAD_INPUT
    dev.set_hamiltonian(h1, h2)  # the handle is still usable
    dev.close()


@pytest.mark.gpu
def test_invalid_mps_and_checkpoints_are_rejected(tmp_path):
    require_gpu()
    from paper_1703_04789_gb300 import SpmpsError
    L, N, D = 6, 6, 12
    labels, tens = inputs.random_mps(L, N, 0, D, 1)
    dev = _spmps(L, N, 0, 0, 4, D)
    dev.set_hubbard(1.0, 4.0)
    t2 = [t.copy() for t in tens]
    nz = np.argwhere(t2[2] != 0)[0]
    t2[2][tuple(nz)] = np.nan
    with pytest.raises(SpmpsError) as ei:
        dev.set_mps(labels, t2, center=0)
    assert ei.value.status == BAD_INPUT
    l2 = [q.copy() for q in labels]
    l2[3] = l2[3][::-1].copy()  # labels out of order
    with pytest.raises(SpmpsError) as ei:
        dev.set_mps(l2, tens, center=0)
    assert ei.value.status == BAD_INPUT
    dev.set_mps(labels, tens, center=0)
    path = str(tmp_path / "ck.bin")
    dev.save(path)
    E0 = dev.energy()
    blob = open(path, "rb").read()
    for name, data in (("truncated", blob[: len(blob) // 2]), ("magic", b"XXXXXXXX" + blob[8:]),
                       ("header", blob[:8] + np.int32(L + 1).tobytes() + blob[12:])):
        p = str(tmp_path / f"{name}.bin")
        open(p, "wb").write(data)
        with pytest.raises(SpmpsError) as ei:
            dev.load(p)
        assert ei.value.status == BAD_INPUT, name
    assert dev.energy() == E0  # a rejected load leaves the state as it was
    dev.load(path)
    assert dev.energy() == E0
    dev.close()


@pytest.mark.gpu
def test_iteration_cap_reports_not_converged_and_finishes_the_sweep():
    require_gpu()
    from paper_1703_04789_gb300 import SpmpsError
    L, N, D = 6, 6, 12
    labels, tens = inputs.random_mps(L, N, 0, D, 2)
    dev = _spmps(L, N, 0, 0, 4, D, dav_max_iter=1)
    dev.set_hubbard(1.0, 4.0)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    E, st = dev.sweep(2)
    assert st == NOT_CONVERGED
    assert np.all(np.isfinite(E)) and E.shape == (2,)
    lab, ts, c = dev.get_mps()
    assert c == 0  # the sweeps ran to the end
    with pytest.raises(SpmpsError) as ei:
        _spmps(L, N, 0, 0, 4, D, dav_max_iter=0)
    assert ei.value.status == BAD_INPUT
    dev.close()


@pytest.mark.gpu
def test_unreachable_spin_gives_singular_metric():
    """S = 3 with four electrons: no state of the sector has that spin, P = 0 and N_eff = 0."""
    require_gpu()
    from paper_1703_04789_gb300 import SpmpsError
    L, N, D = 4, 4, 8
    labels, tens = inputs.random_mps(L, N, 0, D, 1)
    dev = _spmps(L, N, 0, 6, 7, D)
    dev.set_hubbard(1.0, 4.0)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    with pytest.raises(SpmpsError) as ei:
        dev.optimize_step(0, True)
    assert ei.value.status == SINGULAR_METRIC
    dev.close()


@pytest.mark.gpu
def test_tensor_core_wait_limit_gives_timeout_and_frees_tensor_memory():
    require_gpu()
    from paper_1703_04789_gb300 import SpmpsError
    L, N, D = 6, 6, 12
    rng = np.random.default_rng(5)
    params = (0.05 * rng.standard_normal(67329)).astype(np.float32)
    n = 4096
    r, dh, dn = rng.standard_normal(n), rng.standard_normal(n), rng.random(n)
    out = {}
    for polls in (1, 0):
        dev = _spmps(L, N, 0, 0, 4, D, tc_wait_polls=polls)
        dev.set_hubbard(1.0, 4.0)
        dev.mlp_set_params(params)
        if polls == 1:
            with pytest.raises(SpmpsError) as ei:
                dev.mlp_infer(r, dh, dn, -1.0, tensor_cores=True)
            assert ei.value.status == TIMEOUT
            # the context is still usable on the same handle
            out["f32_after_timeout"] = dev.mlp_infer(r, dh, dn, -1.0, tensor_cores=False)
        else:
            out["tc"] = dev.mlp_infer(r, dh, dn, -1.0, tensor_cores=True)
            out["f32"] = dev.mlp_infer(r, dh, dn, -1.0, tensor_cores=False)
        dev.close()
    assert np.array_equal(out["f32_after_timeout"], out["f32"])
    # a later launch allocates tensor memory again on the same SMs: the timed-out CTAs freed theirs
    assert np.abs(out["tc"] - out["f32"]).max() < 2e-2 * max(1.0, np.abs(out["f32"]).max())
