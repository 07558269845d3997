"""The warm-start network's own kernels against the PyTorch-CPU float64
reference (oracle/warm_start_net.py): forward outputs, every parameter's
gradient (autograd), one Adam step, and descent of the loss."""
import numpy as np
import pytest

from oracle import warm_start_net as wn
from paper_1310_6380_gb300 import cells, warmstart

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

NV, MP, KPER = 12, 3, 2
L = 2 * (2 * MP + 1) ** 2


@pytest.fixture(scope="module")
def setup():
    cl = [cells.config3_cell(i)["cell"] for i in (0, 1, 4)]
    pack = warmstart.CellPack(cl)
    rng = np.random.default_rng(7)
    Q = rng.uniform(0, 0.5, (len(cl), KPER, 2))
    V = (rng.standard_normal((len(cl), KPER, 10, L)) +
         1j * rng.standard_normal((len(cl), KPER, 10, L))).astype(np.complex64)
    net = warmstart.WarmStartNet(NV, MP, max_cells=8, max_samples=32, seed=3)
    x = np.stack([wn.encode(c.phase, c.lam, c.mu, c.rho) for c in cl])
    kf = np.stack([wn.kfeatures(Q[c, j], cl[c].lattice == "hex")
                   for c in range(len(cl)) for j in range(KPER)])
    yield cl, pack, Q, V, net, x, kf
    net.close()


def test_forward_matches_reference(setup):
    cl, pack, Q, V, net, x, kf = setup
    p = net.params()
    U = net.predict(pack, Q)                                     # (C, kper, nv, L)
    out = wn.forward(torch.tensor(p.astype(np.float64)), torch.tensor(x), torch.tensor(kf),
                     KPER, NV, MP).numpy()
    ref = out.reshape(len(cl), KPER, NV, L, 2)
    ref = ref[..., 0] + 1j * ref[..., 1]
    err = np.abs(U - ref).max() / np.abs(ref).max()
    assert err < 2e-5, err


def test_gradients_match_autograd(setup):
    cl, pack, Q, V, net, x, kf = setup
    p = net.params()
    loss = net.train_step(pack, Q, V, lr=0.0)
    g = net.grads()
    Vr = V.reshape(len(cl) * KPER, 10, L).transpose(0, 2, 1)
    lref, gref = wn.loss_and_grad(p.astype(np.float64), x, kf, KPER, Vr, NV, MP)
    assert np.allclose(loss, lref, rtol=1e-4, atol=1e-5), (loss, lref)
    o = 0
    for name, shape in wn.layout(NV, MP):
        n = int(np.prod(shape))
        a, b = g[o:o + n].astype(np.float64), gref[o:o + n]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel < 2e-3, (name, rel)
        o += n


def test_adam_step(setup):
    cl, pack, Q, V, net, x, kf = setup
    p0 = net.params()
    net.set_params(p0)                         # resets the moments
    lr = 1e-3
    net.train_step(pack, Q, V, lr=lr)
    g = net.grads().astype(np.float64)
    p1 = net.params().astype(np.float64)
    # first Adam step: m = (1-b1) g, v = (1-b2) g^2, bias-corrected m/sqrt(v) = sign(g)
    m_hat = g
    v_hat = g * g
    want = p0 - lr * m_hat / (np.sqrt(v_hat) + 1e-8)
    assert np.allclose(p1, want, atol=1e-6, rtol=1e-5)
    net.set_params(p0)


def test_training_reduces_loss(setup):
    cl, pack, Q, V, net, x, kf = setup
    p0 = net.params()
    first = net.train_step(pack, Q, V, lr=0.0).mean()
    for _ in range(30):
        net.train_step(pack, Q, V, lr=3e-4)
    last = net.train_step(pack, Q, V, lr=0.0).mean()
    net.set_params(p0)
    assert last < 0.8 * first, (first, last)
