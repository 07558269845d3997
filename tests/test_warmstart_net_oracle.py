"""Pins of the warm-start network reference (oracle/warm_start_net.py):
properties the subspace loss and the periodic convolutions must have, and
autograd gradients against central finite differences."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import warm_start_net as wn  # noqa: E402

NV, MP = 4, 1
L = 2 * (2 * MP + 1) ** 2


def _rand_params(seed, scale=0.05):
    rng = np.random.default_rng(seed)
    n = sum(int(np.prod(s)) for _, s in wn.layout(NV, MP))
    return rng.standard_normal(n) * scale


def _crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_loss_zero_when_prediction_spans_targets():
    rng = np.random.default_rng(0)
    V = torch.tensor(_crand(rng, 3, L, 2))
    U = torch.cat([V, torch.tensor(_crand(rng, 3, L, 2))], dim=2)
    loss = wn.subspace_loss(U, V).numpy()
    assert np.all(np.abs(loss) < 1e-3)          # eps I regularisation only


def test_loss_one_when_orthogonal():
    V = torch.zeros(1, L, 2, dtype=torch.complex128)
    V[0, 0, 0] = 1.0
    V[0, 1, 1] = 1.0j
    U = torch.zeros(1, L, 3, dtype=torch.complex128)
    U[0, 2, 0] = 1.0
    U[0, 3, 1] = 2.0
    U[0, 4, 2] = 1.0 - 1.0j
    assert abs(wn.subspace_loss(U, V).item() - 1.0) < 1e-12


def test_loss_invariant_under_change_of_basis():
    rng = np.random.default_rng(1)
    V = torch.tensor(_crand(rng, 2, L, 3))
    U = torch.tensor(_crand(rng, 2, L, 4)) * 10
    Mx = torch.tensor(_crand(rng, 4, 4))
    a = wn.subspace_loss(U, V).numpy()
    b = wn.subspace_loss(U @ Mx, V).numpy()
    # the eps regularisation is the only basis dependence: tiny for large U
    assert np.allclose(a, b, atol=1e-5)
    assert np.all((a > 0) & (a < 1))


def test_trunk_commutes_with_periodic_shifts():
    rng = np.random.default_rng(2)
    P = wn.unflatten(torch.tensor(_rand_params(3, 0.2)), NV, MP)
    x = torch.tensor(rng.standard_normal((1, 3, 64, 64)))
    # a shift by 16 pixels moves the 4 x 4 pooled grid by one cell
    h = wn.trunk(x, P).reshape(1, 32, 4, 4)
    hs = wn.trunk(torch.roll(x, shifts=(16, 32), dims=(2, 3)), P).reshape(1, 32, 4, 4)
    assert torch.allclose(torch.roll(h, shifts=(1, 2), dims=(2, 3)), hs, atol=1e-10)


def test_autograd_matches_finite_differences():
    rng = np.random.default_rng(4)
    p = _rand_params(5, 0.1)
    x = rng.standard_normal((2, 3, 64, 64))
    kf = rng.standard_normal((4, 7))
    V = _crand(rng, 4, L, 2)
    loss, g = wn.loss_and_grad(p, x, kf, 2, V, NV, MP)
    # coordinates in every layer
    offs, o = [], 0
    for _, shape in wn.layout(NV, MP):
        n = int(np.prod(shape))
        offs += [o, o + n // 2, o + n - 1]
        o += n
    h = 1e-6
    for i in offs:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        lp, _ = wn.loss_and_grad(pp, x, kf, 2, V, NV, MP)
        lm, _ = wn.loss_and_grad(pm, x, kf, 2, V, NV, MP)
        fd = (lp.mean() - lm.mean()) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])
