"""Layout of warm-start coefficients (host logic, no GPU)."""
import numpy as np

from oracle import mixed_variational as mv
from paper_1310_6380_gb300 import warmstart


def test_low_order_index_matches_plane_wave_order():
    M, Mp = 5, 3
    idx = warmstart.low_order_index(M, Mp)
    N = (2 * M + 1) ** 2
    al, be = mv.plane_wave_indices(M)
    alp, bep = mv.plane_wave_indices(Mp)
    Np = (2 * Mp + 1) ** 2
    assert len(idx) == 2 * Np
    for I in range(2):
        sel = idx[I * Np:(I + 1) * Np]
        assert (sel // N == I).all()
        assert np.array_equal(al[sel % N], alp) and np.array_equal(be[sel % N], bep)


def test_truncate_identity_when_mp_equals_m():
    M = 2
    U = (np.arange(3 * 2 * 25) + 1j).reshape(3, 50).astype(np.complex64)
    assert np.array_equal(warmstart.truncate(U, M, M), U)
