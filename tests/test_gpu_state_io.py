"""MPS initialisation (determinant, random) and checkpoint files through the C ABI."""
import os

import numpy as np
import pytest

from oracle import fock
from paper_1703_04789_gb300 import inputs
from tests.gpu_util import require_gpu


def _dev(K, N, twoM, twoS, D, G, **kw):
    from paper_1703_04789_gb300 import Spmps
    d = Spmps(K, N, twoM, twoS, G, D, **kw)
    return d


@pytest.mark.gpu
def test_closed_shell_determinant_energy_and_growth_to_ed():
    """A closed-shell determinant is a singlet, so P|D> = |D> and the projected energy is the
    diagonal element <D|H|D>; two-site sweeps from it then grow the bonds and reach the lowest
    singlet of the sector."""
    require_gpu()
    K, N = 4, 4
    h1, eri, ecore = inputs.synthetic_active_space(K, 5)
    dev = _dev(K, N, 0, 0, 16, 3, dav_tol_r=1e-8)
    dev.set_hamiltonian(h1, eri, ecore)
    occ = [3, 3, 0, 0]
    dev.init_determinant(occ)
    E, nP = dev.energy()
    H, basis = fock.hamiltonian(K, 2, 2, h1, eri, ecore)
    mask = sum(1 << (2 * k) | 1 << (2 * k + 1) for k in range(2))
    j = int(np.nonzero(basis == mask)[0][0])
    assert abs(nP - 1.0) < 1e-12
    assert abs(E - H[j, j]) < 1e-12
    e_ed, _, _ = fock.lowest_spin_state(K, 2, 2, h1, eri, 0, ecore)
    Es, _ = dev.sweep(4)
    assert abs(Es[-1] - e_ed) < 1e-8
    with pytest.raises(Exception):
        dev.init_determinant([3, 3, 1, 0])  # wrong particle number
    dev.close()


@pytest.mark.gpu
def test_random_init_reaches_ed_and_checkpoint_round_trip(tmp_path):
    require_gpu()
    K, N, twoM, twoS, D, G = 6, 6, 0, 2, 64, 4
    h1, eri = inputs.hubbard_chain(K, 1.0, 4.0)
    Na, Nb = inputs.electron_counts(N, twoM)
    e_ed, _, _ = fock.lowest_spin_state(K, Na, Nb, h1, eri, twoS)
    dev = _dev(K, N, twoM, twoS, D, G, dav_tol_r=1e-8)
    dev.set_hubbard(1.0, 4.0)
    dev.init_random(1234)
    E0, nP0 = dev.energy()
    assert np.isfinite(E0) and 0.0 < nP0 <= 1.0 + 1e-12
    Es, _ = dev.sweep(3)
    assert abs(Es[-1] - e_ed) < 1e-8
    path = os.path.join(tmp_path, "state.spmps")
    dev.save(path)
    other = _dev(K, N, twoM, twoS, D, G)
    other.set_hubbard(1.0, 4.0)
    other.load(path)
    a, b = dev.get_mps(), other.get_mps()
    assert a[2] == b[2]
    for la, lb in zip(a[0], b[0]):
        assert np.array_equal(la, lb)
    for ta, tb in zip(a[1], b[1]):
        assert np.array_equal(ta, tb)
    assert abs(other.energy()[0] - dev.energy()[0]) < 1e-12
    wrong = _dev(K, N + 2, twoM, twoS, D, G)
    with pytest.raises(Exception):
        wrong.load(path)
    for d in (dev, other, wrong):
        d.close()
