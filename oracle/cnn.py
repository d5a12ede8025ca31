"""Plain FP64 reference of the learned post-smoother network (oracle; test
infrastructure only).

The paper has no learned component; this network is the build's extension
of the V-cycle (a residual -> error-correction map replacing the finest-level
post-smoothing).  It has three 3x3 convolution layers with zero padding and
no biases, 1 -> C -> C -> 1 channels, ReLU after the first two:
    a1 = relu(W1 * r),  a2 = relu(W2 * a1),  y = W3 * a2
where (W * a)[co, i, j] = sum_{ci, di, dj} W[co, ci, di, dj] a[ci, i+di-1, j+dj-1].
The training loss is the mean squared error 0.5 mean((y - e)^2) over all
samples and pixels.

Parity unpinned by the paper (nothing in it covers a network).  Pins:
central finite differences of the loss, the adjoint identity of the
convolution, and delta-kernel identities (tests/test_oracle_cnn.py).
"""
import numpy as np


def conv3x3(a, W):
    """a: (B, C_in, H, Wd); W: (C_out, C_in, 3, 3) -> (B, C_out, H, Wd), zero padding."""
    B, Ci, H, Wd = a.shape
    ap = np.zeros((B, Ci, H + 2, Wd + 2))
    ap[:, :, 1:-1, 1:-1] = a
    out = np.zeros((B, W.shape[0], H, Wd))
    for di in range(3):
        for dj in range(3):
            patch = ap[:, :, di:di + H, dj:dj + Wd]                   # (B, Ci, H, Wd)
            out += np.einsum("oc,bchw->bohw", W[:, :, di, dj], patch)
    return out


def conv3x3_adjoint(g, W):
    """Adjoint of conv3x3 in its input: g (B, C_out, H, Wd) -> (B, C_in, H, Wd)."""
    B, Co, H, Wd = g.shape
    Ci = W.shape[1]
    out = np.zeros((B, Ci, H + 2, Wd + 2))
    for di in range(3):
        for dj in range(3):
            out[:, :, di:di + H, dj:dj + Wd] += np.einsum("oc,bohw->bchw", W[:, :, di, dj], g)
    return out[:, :, 1:-1, 1:-1]


def conv3x3_weight_grad(a, g):
    """d/dW of sum(g * conv3x3(a, W)): (C_out, C_in, 3, 3)."""
    B, Ci, H, Wd = a.shape
    ap = np.zeros((B, Ci, H + 2, Wd + 2))
    ap[:, :, 1:-1, 1:-1] = a
    dW = np.zeros((g.shape[1], Ci, 3, 3))
    for di in range(3):
        for dj in range(3):
            dW[:, :, di, dj] = np.einsum("bohw,bchw->oc", g, ap[:, :, di:di + H, dj:dj + Wd])
    return dW


def forward(r, Ws):
    """r: (B, H, Wd) residuals; Ws = (W1, W2, W3).  Returns y (B, H, Wd) and the
    intermediate activations."""
    W1, W2, W3 = Ws
    z1 = conv3x3(r[:, None], W1)
    a1 = np.maximum(z1, 0.0)
    z2 = conv3x3(a1, W2)
    a2 = np.maximum(z2, 0.0)
    y = conv3x3(a2, W3)[:, 0]
    return y, (z1, a1, z2, a2)


def loss_and_grads(r, e, Ws):
    """0.5 mean((y - e)^2) and its gradients with respect to W1, W2, W3."""
    W1, W2, W3 = Ws
    y, (z1, a1, z2, a2) = forward(r, Ws)
    n = y.size
    d = y - e
    loss = 0.5 * float(np.sum(d * d)) / n
    gy = (d / n)[:, None]                                  # (B, 1, H, Wd)
    dW3 = conv3x3_weight_grad(a2, gy)
    g2 = conv3x3_adjoint(gy, W3) * (z2 > 0)
    dW2 = conv3x3_weight_grad(a1, g2)
    g1 = conv3x3_adjoint(g2, W2) * (z1 > 0)
    dW1 = conv3x3_weight_grad(r[:, None], g1)
    return loss, (dW1, dW2, dW3)


def adam_step(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma and Ba, 2015) with bias correction; returns (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
