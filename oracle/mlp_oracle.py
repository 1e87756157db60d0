"""Plain FP64 numpy oracle of the scan surrogate (TEST INFRASTRUCTURE ONLY).

The surrogate maps a scan cell's four parameters to its FLI:
    z  = (x - center) / scale                      (4 inputs, normalised)
    h1 = tanh(W1 z + b1)                           (64)
    h2 = tanh(W2 h1 + b2)                          (64)
    y  = w3 . h2 + b3                              (1)
trained by minimising the mean squared error with Adam (Kingma & Ba 2015:
beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected moments).  An ensemble
of K independently initialised members gives a mean and a spread
(max - min over the members).  Only tests/ and bench.py's reference leg may
import this; it shares no code with the CUDA kernels.

Parameter vector layout (P = 4*64 + 64 + 64*64 + 64 + 64 + 1 = 4545):
    W1 (64 x 4, row-major), b1 (64), W2 (64 x 64, row-major: W2[out][in]),
    b2 (64), w3 (64), b3 (1)
"""
import numpy as np

N_IN, N_H = 4, 64
OFF_W1 = 0
OFF_B1 = OFF_W1 + N_H * N_IN
OFF_W2 = OFF_B1 + N_H
OFF_B2 = OFF_W2 + N_H * N_H
OFF_W3 = OFF_B2 + N_H
OFF_B3 = OFF_W3 + N_H
N_PARAMS = OFF_B3 + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[OFF_W1:OFF_B1].reshape(N_H, N_IN), p[OFF_B1:OFF_W2],
            p[OFF_W2:OFF_B2].reshape(N_H, N_H), p[OFF_B2:OFF_W3],
            p[OFF_W3:OFF_B3], p[OFF_B3])


def pack(W1, b1, W2, b2, w3, b3):
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, np.atleast_1d(b3)]).astype(np.float64)


def normalise(x, center, scale):
    return (np.asarray(x, dtype=np.float64) - center) / scale


def forward(p, z):
    """z: (B, 4) normalised inputs.  Returns (y, cache)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    a1 = z @ W1.T + b1
    h1 = np.tanh(a1)
    a2 = h1 @ W2.T + b2
    h2 = np.tanh(a2)
    y = h2 @ w3 + b3
    return y, (z, h1, h2)


def loss_and_grad(p, z, t):
    """Mean squared error over the batch and its gradient wrt p (backprop)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    y, (z, h1, h2) = forward(p, z)
    B = z.shape[0]
    e = y - t
    loss = np.mean(e * e)
    d3 = 2.0 * e / B                       # dL/dy
    gw3 = h2.T @ d3
    gb3 = np.sum(d3)
    d2 = np.outer(d3, w3) * (1.0 - h2 * h2)    # dL/da2
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)           # dL/da1
    gW1 = d1.T @ z
    gb1 = d1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gw3, gb3)


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


GOLDEN_GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 (Steele, Lea & Flood 2014): advance the state by the golden
    gamma and return the output mix of the new state.  Python integers,
    reduced modulo 2**64 after every operation."""
    z = (int(x) + GOLDEN_GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def batch_rows(seed, member, t, n, batch=128):
    """Rows of the minibatch of Adam step t (from 1) of ensemble member
    `member`, drawn with replacement from n rows: row j is
    SM(seed ^ SM((member << 40) ^ ((t - 1) << 8) ^ j)) mod n."""
    out = np.empty(batch, dtype=np.int64)
    for j in range(batch):
        key = ((int(member) << 40) ^ ((int(t) - 1) << 8) ^ j) & MASK64
        out[j] = splitmix64(int(seed) ^ splitmix64(key)) % int(n)
    return out


def ensemble_predict(params, z):
    """params: (K, P).  Returns (mean, spread = max - min) over the members."""
    ys = np.stack([forward(p, z)[0] for p in params])
    return ys.mean(axis=0), ys.max(axis=0) - ys.min(axis=0)


def train(p0, z, t, steps, batch, lr, rng):
    """Plain minibatch Adam (samples drawn with replacement); returns (p, losses)."""
    p = p0.copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    losses = []
    for k in range(1, steps + 1):
        idx = rng.integers(0, z.shape[0], batch)
        loss, g = loss_and_grad(p, z[idx], t[idx])
        p, m, v = adam_step(p, g, m, v, k, lr)
        losses.append(loss)
    return p, np.array(losses)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64:
    bfloat16 keeps the top 16 bits of an IEEE float32."""
    f = np.asarray(x, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(p, z):
    """forward() with the hidden-layer contraction's operands (W2 and h1)
    rounded to bfloat16, as a BF16 tensor-core kernel computes it."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    h1 = np.tanh(z @ W1.T + b1)
    h2 = np.tanh(bf16_round(h1) @ bf16_round(W2).T + b2)
    return h2 @ w3 + b3, (z, h1, h2)


def loss_and_grad_bf16(p, z, t):
    """loss_and_grad() with BF16 operands wherever a BF16 tensor-core kernel
    has them: h1 and W2 in the forward contraction; the hidden-2 error d2 and
    h1 in dL/dW2; d2 and W2 in the error propagated to layer 1; d2 in dL/db2."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    y, (z, h1, h2) = forward_bf16(p, z)
    B = z.shape[0]
    e = y - t
    loss = np.mean(e * e)
    d3 = 2.0 * e / B
    gw3 = h2.T @ d3
    gb3 = np.sum(d3)
    d2 = bf16_round(np.outer(d3, w3) * (1.0 - h2 * h2))
    gW2 = d2.T @ bf16_round(h1)
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ bf16_round(W2)) * (1.0 - h1 * h1)
    gW1 = d1.T @ z
    gb1 = d1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gw3, gb3)
