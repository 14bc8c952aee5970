"""Oracle: the learned schedule's network, loss, gradients and optimiser step,
and the per-box features and targets it is trained on.

Test infrastructure only (see ``oracle/__init__``).  The paper has no learned
part; this module states, in plain FP64 numpy, the small network the library
trains on the GPU to predict per-box term cut-offs of the screen (Sec. 4's
term ranges, narrowed per output box), so the GPU kernels can be checked
against it.

Network (3 hidden layers of H = 128 units, ReLU):
    h1 = R(W1 x + b1), h2 = R(W2 h1 + b2), h3 = R(W3 h2 + b3), y = W4 h3 + b4
with R(z) = fp16(max(z, 0)) when ``fp16=True``: the weights used in the
products are the FP16 roundings of the FP32 master weights, and each hidden
activation is rounded to FP16 after the ReLU (the storage format of the GPU
path); everything else is FP64 here.  ``fp16=False`` is the plain FP64
network (used by the finite-difference pins).

Outputs per box: for each Core/Boundary class S = 0..3 (number of directions
with |t_d| <= 1), three numbers [e_S, lo_S, hi_S]: a logit for "no item of
class S survives the exact screen" and the normalised first / last surviving
term m / (M - 1).  Loss per box:
    sum_S softplus(e_S) - E_S e_S + (1 - E_S) ((lo_S - LO_S)^2 + (hi_S - HI_S)^2)
(binary cross-entropy with logits, squared error on the range when the class
is not empty), averaged over the batch.

Optimiser: Adam (Kingma & Ba) on the FP32 master weights,
beta1 = 0.9, beta2 = 0.999, eps_adam = 1e-8, bias-corrected.

Parity: pinned by central finite differences of the FP64 network (every
weight and bias), by the closed-form loss of the zero network, and by a
hand-derived single-unit case (tests/test_oracle_mlp.py).
"""
import numpy as np

H = 128
N_OUT = 12


def param_shapes(n_in, n_out=N_OUT, hidden=H):
    """Parameter order of the flat vector: W1 (H, n_in), b1, W2 (H, H), b2,
    W3 (H, H), b3, W4 (n_out, H), b4 (row-major)."""
    return [(hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (hidden, hidden), (hidden,),
            (n_out, hidden), (n_out,)]


def unflatten(theta, n_in, n_out=N_OUT, hidden=H):
    out, o = [], 0
    for shp in param_shapes(n_in, n_out, hidden):
        size = int(np.prod(shp))
        out.append(np.asarray(theta[o:o + size], dtype=np.float64).reshape(shp))
        o += size
    return out


def flatten(params):
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in params])


def fp16(a):
    return np.asarray(a, dtype=np.float64).astype(np.float16).astype(np.float64)


def forward(params, x, fp16_storage=True):
    """Returns (y, cache): y (n, n_out) and the activations the backward pass
    needs."""
    W1, b1, W2, b2, W3, b3, W4, b4 = params
    q = fp16 if fp16_storage else (lambda a: np.asarray(a, dtype=np.float64))
    Ws = [q(W1), q(W2), q(W3), q(W4)]
    h0 = np.asarray(x, dtype=np.float64)
    z1 = h0 @ Ws[0].T + b1
    h1 = q(np.maximum(z1, 0.0))
    z2 = h1 @ Ws[1].T + b2
    h2 = q(np.maximum(z2, 0.0))
    z3 = h2 @ Ws[2].T + b3
    h3 = q(np.maximum(z3, 0.0))
    y = h3 @ Ws[3].T + b4
    return y, (Ws, h0, h1, h2, h3)


def loss_and_dy(y, target):
    """Mean loss over the rows and dL/dy.  target (n, 12) holds per class
    [E_S, LO_S, HI_S] with E_S in {0, 1}."""
    n = y.shape[0]
    L = 0.0
    dy = np.zeros_like(y)
    for S in range(4):
        e, lo, hi = y[:, 3 * S], y[:, 3 * S + 1], y[:, 3 * S + 2]
        E, LO, HI = target[:, 3 * S], target[:, 3 * S + 1], target[:, 3 * S + 2]
        sp = np.logaddexp(0.0, e)                       # softplus
        L += float(np.sum(sp - E * e + (1.0 - E) * ((lo - LO) ** 2 + (hi - HI) ** 2)))
        dy[:, 3 * S] = 1.0 / (1.0 + np.exp(-e)) - E
        dy[:, 3 * S + 1] = 2.0 * (1.0 - E) * (lo - LO)
        dy[:, 3 * S + 2] = 2.0 * (1.0 - E) * (hi - HI)
    return L / n, dy / n


def backward(params, cache, dy):
    """Gradients of the mean loss with respect to every parameter (the
    products use the same weights as the forward pass)."""
    Ws, h0, h1, h2, h3 = cache
    gW4 = dy.T @ h3
    gb4 = dy.sum(axis=0)
    d3 = (dy @ Ws[3]) * (h3 > 0)
    gW3 = d3.T @ h2
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ Ws[2]) * (h2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ Ws[1]) * (h1 > 0)
    gW1 = d1.T @ h0
    gb1 = d1.sum(axis=0)
    return [gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4]


def loss_grad(theta, x, target, n_in, fp16_storage=True, hidden=H):
    params = unflatten(theta, n_in, N_OUT, hidden)
    y, cache = forward(params, x, fp16_storage)
    L, dy = loss_and_dy(y, target)
    return L, flatten(backward(params, cache, dy))


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
