"""Reference of the learned warm-start network, for the tests only.

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline may import this module; the library never calls it.

The paper has no learned component; the network is an addition that
predicts a starting subspace for the block eigen-solver.  This module
writes the same network and loss in plain PyTorch CPU operations in float64
(torch.nn.functional conv2d with circular padding, avg_pool2d, linear,
complex linear algebra), and takes gradients from autograd, so that the
hand-written forward and backward kernels can be checked against it.

Parameter layout (one flat vector, as the library's): for each of the four
convolutions (3->16, 16->32, 32->32, 32->32) its weights [co][ci][3][3] then
biases [co]; then for each dense layer (519->512, 512->512, 512->out) its
weights [out][in] then biases [out].

Parity pins (tests/test_warmstart_net_oracle.py): the loss is 0 when the
prediction spans the targets, 1 when it is orthogonal to them, invariant
under a change of basis of the prediction; autograd gradients agree with
central finite differences of the loss; the convolutional trunk commutes
with periodic shifts of the cell by multiples of 16 pixels (the pooling
stride).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CONV = [(3, 16), (16, 32), (32, 32), (32, 32)]
FEAT, KF, HID = 512, 7, 512
EPS = 1e-4


def n_out(nvec: int, Mp: int) -> int:
    return nvec * 2 * (2 * Mp + 1) ** 2 * 2


def layout(nvec: int, Mp: int):
    """[(name, shape)] in the order of the flat parameter vector."""
    out = []
    for l, (ci, co) in enumerate(CONV):
        out += [(f"conv{l}.w", (co, ci, 3, 3)), (f"conv{l}.b", (co,))]
    dims = [(FEAT + KF, HID), (HID, HID), (HID, n_out(nvec, Mp))]
    for l, (di, do) in enumerate(dims):
        out += [(f"dense{l}.w", (do, di)), (f"dense{l}.b", (do,))]
    return out


def unflatten(p, nvec: int, Mp: int):
    params, o = {}, 0
    for name, shape in layout(nvec, Mp):
        n = int(np.prod(shape))
        params[name] = p[o:o + n].reshape(shape)
        o += n
    assert o == p.numel()
    return params


def encode(phase, lam, mu, rho):
    """(3, 64, 64): standardised log(lam + 2 mu), log mu, log rho of every pixel."""
    ph = np.asarray(phase, np.int64)
    lam, mu, rho = (np.asarray(v, float)[ph] for v in (lam, mu, rho))
    return np.stack([(np.log(lam + 2 * mu) - 3.5) / 1.0, (np.log(mu) - 2.2) / 1.2,
                     (np.log(rho) - 1.0) / 0.6])


def kfeatures(Q, hexagonal: bool):
    q1, q2 = float(Q[0]), float(Q[1])
    return np.array([q1, q2, np.cos(2 * np.pi * q1), np.sin(2 * np.pi * q1),
                     np.cos(2 * np.pi * q2), np.sin(2 * np.pi * q2), 1.0 if hexagonal else 0.0])


def trunk(x, P):
    """x: (cells, 3, 64, 64) -> (cells, 512)."""
    h = x
    for l in range(len(CONV)):
        h = F.conv2d(F.pad(h, (1, 1, 1, 1), mode="circular"), P[f"conv{l}.w"], P[f"conv{l}.b"])
        h = F.avg_pool2d(F.relu(h), 2)
    return h.flatten(1)


def head(feat, kf, kper, P):
    """feat (cells, 512), kf (cells*kper, 7) -> (cells*kper, out)."""
    h = torch.cat([feat.repeat_interleave(kper, 0), kf], 1)
    h = F.relu(F.linear(h, P["dense0.w"], P["dense0.b"]))
    h = F.relu(F.linear(h, P["dense1.w"], P["dense1.b"]))
    return F.linear(h, P["dense2.w"], P["dense2.b"])


def as_complex_block(out, nvec, L):
    """(samples, nvec*L*2) -> (samples, L, nvec) complex."""
    o = out.reshape(out.shape[0], nvec, L, 2)
    return torch.complex(o[..., 0], o[..., 1]).transpose(1, 2)


def subspace_loss(U, V):
    """Per-sample (||V||^2 - Re tr(B^H (U^H U + eps I)^-1 B)) / ||V||^2, B = U^H V."""
    nv = U.shape[-1]
    G = U.conj().transpose(-2, -1) @ U + EPS * torch.eye(nv, dtype=U.dtype)
    B = U.conj().transpose(-2, -1) @ V
    Fm = torch.linalg.solve(G, B)
    cap = torch.real(torch.einsum("sij,sij->s", B.conj(), Fm))
    v2 = torch.sum(torch.abs(V) ** 2, dim=(-2, -1))
    return (v2 - cap) / v2


def forward(p, x, kf, kper, nvec, Mp):
    P = unflatten(p, nvec, Mp)
    return head(trunk(x, P), kf, kper, P)


def loss_and_grad(p_np, x_np, kf_np, kper, V_np, nvec, Mp):
    """Mean loss over samples and its gradient (flat, float64) by autograd."""
    p = torch.tensor(np.asarray(p_np, np.float64), requires_grad=True)
    x = torch.tensor(np.asarray(x_np, np.float64))
    kf = torch.tensor(np.asarray(kf_np, np.float64))
    V = torch.tensor(np.asarray(V_np, np.complex128))
    L = 2 * (2 * Mp + 1) ** 2
    U = as_complex_block(forward(p, x, kf, kper, nvec, Mp), nvec, L)
    losses = subspace_loss(U, V)
    loss = losses.mean()
    loss.backward()
    return losses.detach().numpy(), p.grad.numpy()
