"""FP64-accurate block products on the tensor cores (option fp64_tensor_cores): parity with the oracle.

Every FP64 block product of phases A and C of the projected action (H and N) is computed from
exact products of 8-bit digits (error-free splitting, Ozaki et al. 2012) on tcgen05.mma kind::f16
with exact FP32 level sums.  The error per K stage is of the order of 32 * 2^-55 of the product of
the line maxima, the size of FP64 rounding, so the bound against the oracle is the FP64 one:
1e-10 relative to max |y| (max |z|), element by element.  The difference to the library's own FP64
pipe must be nonzero (the split path ran) and at the level of FP64 rounding.
"""
import numpy as np
import pytest

from oracle import mpo as M, mps as S
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import masked_random_two_site, require_gpu

RTOL = 1e-10
OZAKI_KIND = 9  # spmps_kernel_stats kind of the split-product GEMM launches


def _pair(P, L, N, twoM, twoS, G, D, ham):
    from paper_1703_04789_gb300 import Spmps
    out = []
    for tc in (False, True):
        dev = Spmps(L, N, twoM, twoS, G, D, fp64_tensor_cores=tc)
        ham(dev)
        dev.set_mps(P.mps.labels, P.mps.A, center=0)
        out.append(dev)
    return out


def _check_site(P, devs, k, rng):
    ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
    lay = devs[0].x_layout(k)
    x = masked_random_two_site(ql, qr, rng)
    y_ref, z_ref = P.apply(x, k)
    xv = devs[0].pack(x, lay, ql, qr)
    y64, z64 = devs[0].apply_heff_host(k, xv)
    yv, zv = devs[1].apply_heff_host(k, xv)
    y = devs[1].unpack(yv, lay, ql, qr)
    z = devs[1].unpack(zv, lay, ql, qr)
    sy, sz = max(1.0, np.abs(y_ref).max()), max(1.0, np.abs(z_ref).max())
    assert np.abs(y - y_ref).max() <= RTOL * sy, (k, np.abs(y - y_ref).max())
    assert np.abs(z - z_ref).max() <= RTOL * sz, (k, np.abs(z - z_ref).max())
    # same numbers as the FP64 pipe to FP64 rounding
    assert np.abs(yv - y64).max() <= 1e-12 * sy and np.abs(zv - z64).max() <= 1e-12 * sz
    return np.abs(yv - y64).max() + np.abs(zv - z64).max()


@pytest.mark.gpu
@pytest.mark.parametrize("case", [
    # L, N, 2M, 2S, D, n_beta, seed, U
    (6, 6, 0, 0, 16, 4, 2, 4.0),
    (7, 7, 1, 3, 20, 4, 3, 2.5),
    (8, 8, 0, 0, 32, 5, 1, 4.0),     # the L=8, D=32, n_beta=5 workload
    (6, 5, -1, 1, 12, 3, 5, 4.0),    # negative M, odd N
])
def test_hubbard_action_matches_oracle_every_site(case):
    require_gpu()
    L, N, twoM, twoS, D, G, seed, U = case
    labels, tens = inputs.random_mps(L, N, twoM, D, seed)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, U), twoS, twoM, G)
    devs = _pair(P, L, N, twoM, twoS, G, D, lambda d: d.set_hubbard(1.0, U))
    devs[1].profile(True)
    rng = np.random.default_rng(seed + 3000)
    P.build_left(L - 2)
    diff = sum(_check_site(P, devs, k, rng) for k in range(L - 1))
    assert devs[1].kernel_stats(OZAKI_KIND)["launches"] > 0
    assert diff > 0.0  # the split products ran (they round differently from the FP64 pipe)
    for d in devs:
        d.close()


@pytest.mark.gpu
@pytest.mark.parametrize("case", [(5, 6, 2, 2, 12, 4, 2), (6, 6, 0, 0, 12, 4, 4)])
def test_ab_initio_action_matches_oracle_every_site(case):
    """Complementary-operator MPO: phase C reduces over many channel segments."""
    require_gpu()
    K, N, twoM, twoS, D, G, seed = case
    h1, eri, ecore = inputs.synthetic_active_space(K, seed)
    labels, tens = inputs.random_mps(K, N, twoM, D, seed)
    P = S.prepare(labels, tens, M.ab_initio_mpo(h1, eri, ecore), twoS, twoM, G)
    devs = _pair(P, K, N, twoM, twoS, G, D, lambda d: d.set_hamiltonian(h1, eri, ecore))
    rng = np.random.default_rng(seed + 4000)
    P.build_left(K - 2)
    for k in range(K - 1):
        _check_site(P, devs, k, rng)
    for d in devs:
        d.close()


@pytest.mark.gpu
@pytest.mark.parametrize("twoM,twoS", [(0, 0), (2, 2)])
def test_full_size_action_sampled_rows(twoM, twoS):
    """Hubbard L=24, half filling, D=256, n_beta=8, middle site: sampled bra rows against the
    oracle, the whole output against the FP64 pipe, and the symmetry of H_eff and N_eff."""
    require_gpu()
    L, N, D, G, U = 24, 24, 256, 8, 4.0
    labels, tens = inputs.random_mps(L, N, twoM, D, 2)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, U), twoS, twoM, G)
    devs = _pair(P, L, N, twoM, twoS, G, D, lambda d: d.set_hubbard(1.0, U))
    k = L // 2 - 1
    P.build_left(k)
    ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
    rng = np.random.default_rng(7)
    x = masked_random_two_site(ql, qr, rng)
    lay = devs[1].x_layout(k)
    x1 = devs[1].pack(x, lay, ql, qr)
    yv, zv = devs[1].apply_heff_host(k, x1)
    y64, z64 = devs[0].apply_heff_host(k, x1)
    rows = sorted(set(rng.choice(ql.shape[0], size=12, replace=False).tolist() + [0, ql.shape[0] - 1]))
    y_ref, z_ref = P.apply_rows(x, k, rows)
    y = devs[1].unpack(yv, lay, ql, qr)
    z = devs[1].unpack(zv, lay, ql, qr)
    sy, sz = max(1.0, np.abs(y_ref).max()), max(1.0, np.abs(z_ref).max())
    assert np.abs(y[rows] - y_ref).max() <= RTOL * sy
    assert np.abs(z[rows] - z_ref).max() <= RTOL * sz
    assert 0.0 < np.abs(yv - y64).max() <= 1e-12 * max(1.0, np.abs(y64).max())
    assert np.abs(zv - z64).max() <= 1e-12 * max(1.0, np.abs(z64).max())
    x2 = devs[1].pack(masked_random_two_site(ql, qr, rng), lay, ql, qr)
    y2, z2 = devs[1].apply_heff_host(k, x2)
    assert abs(x1 @ y2 - x2 @ yv) <= 1e-11 * np.linalg.norm(x1) * np.linalg.norm(y2)
    assert abs(x1 @ z2 - x2 @ zv) <= 1e-11 * np.linalg.norm(x1) * np.linalg.norm(z2)
    for d in devs:
        d.close()


@pytest.mark.gpu
@pytest.mark.parametrize("case", [(8, 8, 0, 0, 32, 5, 1), (7, 7, 1, 3, 20, 4, 2)])
def test_step_theta_matches_oracle(case):
    """The lowest generalised eigenvalue of one two-site step (unique) equals the oracle's."""
    require_gpu()
    from paper_1703_04789_gb300 import Spmps
    L, N, twoM, twoS, D, G, seed = case
    labels, tens = inputs.random_mps(L, N, twoM, D, seed)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, 4.0), twoS, twoM, G)
    dev = Spmps(L, N, twoM, twoS, G, D, dav_tol_r=1e-9, dav_max_iter=400, fp64_tensor_cores=True)
    dev.set_hubbard(1.0, 4.0)
    dev.set_mps(P.mps.labels, P.mps.A, center=0)
    th, it = dev.optimize_step(0, True)
    mask = S.two_site_mask(P.mps.labels[0], P.mps.labels[2])
    dh, dn = P.diagonal(0)
    res = S.davidson(lambda v: P.apply(v, 0), P.two_site(0), dh, dn, mask, tol_r=1e-9, max_iter=400)
    assert res.converged
    assert abs(th - res.theta) < 1e-9 * max(1.0, abs(res.theta)), (th, res.theta, it)
    dev.close()


@pytest.mark.gpu
def test_untruncated_sweeps_reach_ed():
    """L=8 half filling, D=256 (no truncation), n_beta=5, every action on the split products:
    the sweep energy equals the lowest S=0 eigenvalue of the 4900-dimensional sector.  Truncated
    sweeps are not compared with the FP64 pipe: their trajectories depend on rounding (steps
    stopped at the iteration cap, nearly equal singular values at the truncation), and at L=8,
    D=32 two sweeps from the same MPS parted by 1.6e-5."""
    require_gpu()
    from oracle import fock
    from paper_1703_04789_gb300 import Spmps
    L, N, D, G = 8, 8, 256, 5
    h1, eri = inputs.hubbard_chain(L, 1.0, 4.0)
    e_ed, _, _ = fock.lowest_spin_state(L, 4, 4, h1, eri, 0)
    labels, tens = inputs.random_mps(L, N, 0, D, 1)
    dev = Spmps(L, N, 0, 0, G, D, dav_tol_r=1e-8, dav_max_iter=400, fp64_tensor_cores=True)
    dev.set_hubbard(1.0, 4.0)
    dev.set_mps(labels, tens, center=0)
    dev.canonicalize()
    dev.profile(True)
    E, _ = dev.sweep(4)
    assert abs(E[-1] - e_ed) < 1e-10, (E, e_ed)
    assert abs(dev.expect_s2()) < 1e-9
    assert dev.kernel_stats(OZAKI_KIND)["launches"] > 0
    dev.close()
