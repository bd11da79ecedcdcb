"""Parity of the CUDA projected action (spmps_apply_heff) with the CPU oracle.

y = sum_g c_g [H exp(-i b_g S_y)]_eff x and z = sum_g c_g [exp(-i b_g S_y)]_eff x
(Eq. geproblem, Fig. spmpsOpt) on the same seeded MPS and the same x, element by element.
FP64 path: the bound is 1e-10 relative to max |y| (the FP64 contraction differs from the
oracle only in summation order).
"""
import numpy as np
import pytest

from oracle import mpo as M, mps as S, quadrature as Q
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import masked_random_two_site, require_gpu

RTOL = 1e-10

CASES = [
    # L, N, 2M, 2S, D, n_beta, seed, U
    (4, 4, 0, 0, 8, 2, 1, 4.0),
    (6, 6, 0, 0, 16, 4, 2, 4.0),
    (7, 7, 1, 3, 20, 4, 3, 2.5),
    (8, 8, 0, 0, 32, 5, 1, 4.0),     # the L=8, D=32, n_beta=5 workload
    (8, 8, 2, 2, 24, 5, 4, 8.0),
    (6, 5, -1, 1, 12, 3, 5, 4.0),    # negative M, odd N
    (5, 10, 0, 0, 4, 1, 6, 4.0),     # full band: one state, n_beta = 1
]


def _setup(L, N, twoM, twoS, D, G, seed, U, batched=True):
    from paper_1703_04789_gb300 import Spmps
    labels, tens = inputs.random_mps(L, N, twoM, D, seed)
    P = S.prepare(labels, tens, M.hubbard_mpo(L, 1.0, U), twoS, twoM, G)
    dev = Spmps(L, N, twoM, twoS, G, D, batched=batched)
    dev.set_hubbard(1.0, U)
    dev.set_mps(P.mps.labels, P.mps.A, center=0)
    return P, dev


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES)
def test_apply_matches_oracle_every_site(case):
    require_gpu()
    L, N, twoM, twoS, D, G, seed, U = case
    P, dev = _setup(*case)
    b, c = dev.quadrature()
    assert np.allclose(b, P.beta, atol=1e-14) and np.allclose(c, P.c, atol=1e-14)
    rng = np.random.default_rng(seed + 1000)
    P.build_left(L - 2)
    for k in range(L - 1):
        ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
        lay = dev.x_layout(k)
        x = masked_random_two_site(ql, qr, rng)
        y_ref, z_ref = P.apply(x, k)
        xv = dev.pack(x, lay, ql, qr)
        assert abs(np.linalg.norm(xv) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
        yv, zv = dev.apply_heff_host(k, xv)
        y = dev.unpack(yv, lay, ql, qr)
        z = dev.unpack(zv, lay, ql, qr)
        sy = max(1.0, np.abs(y_ref).max())
        sz = max(1.0, np.abs(z_ref).max())
        assert np.abs(y - y_ref).max() <= RTOL * sy, (k, np.abs(y - y_ref).max())
        assert np.abs(z - z_ref).max() <= RTOL * sz, (k, np.abs(z - z_ref).max())
    dev.close()


@pytest.mark.gpu
def test_device_pointer_apply_and_unbatched_launches_agree():
    require_gpu()
    import torch
    case = (8, 8, 0, 0, 32, 5, 1, 4.0)
    P, dev = _setup(*case)
    _, dev1 = _setup(*case, batched=False)
    k = 3
    lay = dev.x_layout(k)
    rng = np.random.default_rng(0)
    xv = rng.standard_normal(lay["n_x"])
    x = torch.tensor(xv, device="cuda")
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    stream = torch.cuda.Stream()
    dev.apply_heff(k, x, y, z, stream=stream)
    stream.synchronize()
    y1, z1 = dev1.apply_heff_host(k, xv)
    assert np.array_equal(y.cpu().numpy(), y1) and np.array_equal(z.cpu().numpy(), z1)
    # y only / z only calls give the same numbers
    y2 = torch.empty_like(x)
    dev.apply_heff(k, x, y2, None)
    torch.cuda.synchronize()
    assert torch.equal(y2, y)
    dev.close()
    dev1.close()


@pytest.mark.gpu
@pytest.mark.parametrize("case", [(6, 6, 0, 0, 16, 4, 2, 4.0), (8, 8, 2, 2, 24, 5, 4, 8.0)])
def test_energy_functional_matches_oracle(case):
    require_gpu()
    P, dev = _setup(*case)
    E, nP = dev.energy()
    E_ref, nP_ref = P.energy(0)
    assert abs(E - E_ref) < 1e-11 * max(1.0, abs(E_ref))
    assert abs(nP - nP_ref) < 1e-12
    dev.close()


@pytest.mark.gpu
@pytest.mark.parametrize("twoM,twoS", [(0, 0), (2, 2)])
def test_full_size_apply_sampled_rows(twoM, twoS):
    """Hubbard L=24, half filling, D=256, n_beta=8 (the plain-vs-batched workload): the oracle
    computes y and z on sampled bra rows of the middle site; every GPU output entry of those
    rows must match."""
    require_gpu()
    L, N, D, G, U = 24, 24, 256, 8, 4.0
    P, dev = _setup(L, N, twoM, twoS, D, G, 2, U)
    k = L // 2 - 1
    P.build_left(k)
    ql, qr = P.mps.labels[k], P.mps.labels[k + 2]
    rng = np.random.default_rng(7)
    x = masked_random_two_site(ql, qr, rng)
    lay = dev.x_layout(k)
    yv, zv = dev.apply_heff_host(k, dev.pack(x, lay, ql, qr))
    y = dev.unpack(yv, lay, ql, qr)
    z = dev.unpack(zv, lay, ql, qr)
    rows = sorted(set(rng.choice(ql.shape[0], size=12, replace=False).tolist() + [0, ql.shape[0] - 1]))
    y_ref, z_ref = P.apply_rows(x, k, rows)
    sy = max(1.0, np.abs(y_ref).max())
    sz = max(1.0, np.abs(z_ref).max())
    assert np.abs(y[rows] - y_ref).max() <= RTOL * sy
    assert np.abs(z[rows] - z_ref).max() <= RTOL * sz
    # properties on the whole output: symmetry of H_eff and N_eff, 0 <= x N x <= |x|^2
    x2 = dev.pack(masked_random_two_site(ql, qr, rng), lay, ql, qr)
    x1 = dev.pack(x, lay, ql, qr)
    y2, z2 = dev.apply_heff_host(k, x2)
    assert abs(x1 @ y2 - x2 @ yv) <= 1e-11 * np.linalg.norm(x1) * np.linalg.norm(y2)
    assert abs(x1 @ z2 - x2 @ zv) <= 1e-11 * np.linalg.norm(x1) * np.linalg.norm(z2)
    assert -1e-12 <= x1 @ zv <= (1 + 1e-12) * (x1 @ x1)
    dev.close()


@pytest.mark.gpu
def test_planner_flop_count_matches_independent_count():
    """The algorithmic flop count reported by the library equals the count derived from the
    block structure alone (used by the CPU-baseline leg of bench.py)."""
    require_gpu()
    import bench
    from paper_1703_04789_gb300 import Spmps
    L, N, D, G = 10, 10, 40, 4
    labels, tens = inputs.random_mps(L, N, 0, D, 1)
    dev = Spmps(L, N, 0, 0, G, D)
    dev.set_hubbard(1.0, 4.0)
    dev.set_mps(labels, tens, center=0)
    for k in (0, 4, 8):
        lib = float(dev.apply_flops(k).sum())
        ref = bench._count_apply_flops(inputs.mps_structure(L, N, 0, D), k, M.hubbard_mpo(L, 1.0, 4.0), G, 0, 0)
        assert abs(lib - ref) <= 1e-9 * ref, (k, lib, ref)
    dev.close()


@pytest.mark.gpu
def test_autotuned_tiles_give_the_same_action():
    """The autotuner only changes tile shapes (summation order): the action agrees with the
    default tiling to rounding, at every site."""
    require_gpu()
    case = (8, 8, 0, 0, 32, 5, 1, 4.0)
    from paper_1703_04789_gb300 import Spmps
    L, N, twoM, twoS, D, G, seed, U = case
    P, dev = _setup(*case)
    tuned = Spmps(L, N, twoM, twoS, G, D, autotune=True)
    tuned.set_hubbard(1.0, U)
    tuned.set_mps(P.mps.labels, P.mps.A, center=0)
    rng = np.random.default_rng(7)
    for k in range(L - 1):
        xv = rng.standard_normal(dev.x_layout(k)["n_x"])
        y0, z0 = dev.apply_heff_host(k, xv)
        y1, z1 = tuned.apply_heff_host(k, xv)
        assert np.abs(y1 - y0).max() <= 1e-12 * max(1.0, np.abs(y0).max())
        assert np.abs(z1 - z0).max() <= 1e-12 * max(1.0, np.abs(z0).max())
    dev.close()
    tuned.close()
