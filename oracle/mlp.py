"""Oracle for the learned-guess network (test infrastructure): the same MLP
(40 -> 256 -> 256 -> 1472, SiLU, per-head masked mean-squared error) in
plain FP64 numpy, forward and backward by the chain rule, used to check the
GPU gradients.  Parameter layout: W1 (256x40), b1, W2 (256x256), b2,
W3 (1472x256), b3, flattened in that order."""
import numpy as np

IN, H, OUT = 40, 256, 1472
HEAD_OFF = [0, 36, 661, 697, 847, 1472]


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = []
    for shape in [(H, IN), (H,), (H, H), (H,), (OUT, H), (OUT,)]:
        n = int(np.prod(shape))
        out.append(p[o:o + n].reshape(shape))
        o += n
    return out


def mask(head):
    M = np.zeros((len(head), OUT))
    for r, h in enumerate(head):
        M[r, HEAD_OFF[h]:HEAD_OFF[h + 1]] = 1.0
    return M


def loss_and_grad(p, X, T, head):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    sig = lambda z: 1.0 / (1.0 + np.exp(-z))
    z1 = X @ W1.T + b1
    h1 = z1 * sig(z1)
    z2 = h1 @ W2.T + b2
    h2 = z2 * sig(z2)
    Y = h2 @ W3.T + b3
    M = mask(head)
    cnt = M.sum()
    d = (Y - T) * M
    loss = float((d * d).sum() / cnt)
    dY = 2.0 * d / cnt
    dsilu = lambda z: sig(z) * (1.0 + z * (1.0 - sig(z)))
    gW3 = dY.T @ h2
    gb3 = dY.sum(0)
    d2 = (dY @ W3) * dsilu(z2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * dsilu(z1)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
