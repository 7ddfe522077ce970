"""Oracle of the flow-curve surrogate: a 4-layer perceptron 5 -> 128 -> 128 -> 128 -> 2
with tanh hidden activations, in FP64 (numpy).

TEST INFRASTRUCTURE ONLY.  The paper has no learned component; this is the
plain definition the CUDA BF16 kernels are checked against:
  inputs  x = (log S, G_AA1, G_AA2, G_AB, tau), normalised per column to
          z = (x - center) / half_range  (center/half_range of the training box)
  h1 = tanh(W1 z + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3),
  out = W4 h3 + b4:  out[0] = normalised stress, out[1] = yielded logit
  loss = mean_b (out0 - t0)^2 + lam * mean_b BCE(out1, label)
         BCE(z, y) = max(z, 0) - z y + log(1 + exp(-|z|))
  Adam (Kingma and Ba 2015) on every parameter with bias correction.
Weights W_l are [out, in] (row = output unit).
"""
import numpy as np

SIZES = (5, 128, 128, 128, 2)


def param_shapes(sizes=SIZES):
    return [((sizes[l + 1], sizes[l]), (sizes[l + 1],)) for l in range(len(sizes) - 1)]


def init_params(seed=0, sizes=SIZES):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases from a seeded
    generator (numpy PCG64); returns a list [(W1, b1), ...]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ps = []
    for (wo, wi), (bo,) in param_shapes(sizes):
        a = 1.0 / np.sqrt(wi)
        ps.append((rng.uniform(-a, a, size=(wo, wi)), rng.uniform(-a, a, size=(bo,))))
    return ps


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(vec, sizes=SIZES):
    out, k = [], 0
    for (wo, wi), (bo,) in param_shapes(sizes):
        W = vec[k:k + wo * wi].reshape(wo, wi)
        k += wo * wi
        b = vec[k:k + bo]
        k += bo
        out.append((W, b))
    assert k == vec.size
    return out


def normalise(x, center, half_range):
    return (np.asarray(x, dtype=np.float64) - center) / half_range


def forward(params, z):
    """Returns (out [B,2], list of activations [z, h1, h2, h3])."""
    acts = [z]
    h = z
    for l, (W, b) in enumerate(params):
        a = h @ W.T + b
        h = np.tanh(a) if l < len(params) - 1 else a
        acts.append(h)
    return h, acts[:-1]


def bce_with_logits(z, y):
    return np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z)))


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def loss(params, z, t_sigma, label, lam=1.0):
    out, _ = forward(params, z)
    B = z.shape[0]
    mse = np.sum((out[:, 0] - t_sigma) ** 2) / B
    bce = np.sum(bce_with_logits(out[:, 1], label)) / B
    return mse + lam * bce


def gradients(params, z, t_sigma, label, lam=1.0):
    """Analytic gradients (backpropagation) of loss(); list [(dW1, db1), ...]."""
    out, acts = forward(params, z)
    B = z.shape[0]
    d = np.zeros_like(out)
    d[:, 0] = 2.0 * (out[:, 0] - t_sigma) / B
    d[:, 1] = lam * (sigmoid(out[:, 1]) - label) / B
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        h_in = acts[l]
        grads[l] = (d.T @ h_in, d.sum(axis=0))
        if l > 0:
            d = (d @ W) * (1.0 - acts[l] ** 2)  # through tanh of layer l-1's output
    return grads


class Adam:
    def __init__(self, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, w, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return w - self.lr * mh / (np.sqrt(vh) + self.eps)
