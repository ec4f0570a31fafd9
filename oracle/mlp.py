"""Learned rank seed of ADC2: node features and the rank model, plain numpy.

Test infrastructure only (see the package docstring).

The paper fixes the rank of an HSS block with eq. (bounds) (Sec. 4.1); the
learned seed replaces that first guess by a small regression model and keeps
the estimate as the fallback.  Nothing here is in the paper: the model and
its features are defined by the library's header and restated below.

  bf16_round     round-to-nearest-even of float32 values to bfloat16 (8-bit
                 significand) by the integer add-and-truncate method     [pinned: torch's
                                                                          bfloat16 cast, hand ties]
  unpack         parameter layout W1[64][7] b1 W2[64][64] b2 w3[64] b3     [pinned: size]
  forward        7 -> 64 -> 64 -> 1 ReLU network; with bf16=True the
                 weights, the standardised input and the hidden activations
                 are rounded to bfloat16 as the device model stores them,
                 sums in float64                                         [pinned: closed-form
                                                                          network y = sum |x| + c]
  loss_grad      0.5 mean (y - t)^2 and its gradient by back-propagation
                 (rounding passed straight through)                      [pinned: central
                                                                          differences, bf16=False]
  adam_step      Adam (Kingma and Ba, ICLR 2015) with bias correction     [pinned: first step
                                                                          moves by lr sign(g)]
  node_features  the 7 features of a node [s0, s1)                      [pinned: hand example]

Feature definitions (K deflated poles d, gaps gamma_i = lambda_i - d_i,
mu_i = d_{i+1} - lambda_i, Loewner vector uhat; spread = lambda_K - d_1):
  0 log2(s1 - s0)
  1 log10(min gap / spread) over gamma_i (i in the node) and mu_i (i in the
    node, i < K - 1)
  2 log10(median gap / spread), the lower median ((c+1)/2-th smallest)
  3 log10(dist / spread), dist = min over the node's inner boundaries b of
    (d_b - d_{b-1}) + gamma_b (the one-sided distance of Sec. 4.1), spread
    when the node has none
  4 log10(sum of uhat_i^2 over the node)
  5 (n - K) / n
  6 log2(K)
The device takes the median from a histogram (bin centre, 0.025 decades); the
oracle takes the exact order statistic, so feature 2 agrees to half a bin.
"""
import numpy as np

IN, H = 7, 64
OFF_B1 = H * IN
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H
NPARAM = OFF_B3 + 1


def bf16_round(x):
    """float32(x) rounded to the nearest bfloat16 (ties to even), as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    bits = (bits + 0x7FFF + lsb) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    assert p.shape == (NPARAM,)
    return (p[:OFF_B1].reshape(H, IN), p[OFF_B1:OFF_W2], p[OFF_W2:OFF_B2].reshape(H, H),
            p[OFF_B2:OFF_W3], p[OFF_W3:OFF_B3], p[OFF_B3])


def _standardise(X, mean, std, bf16):
    if bf16:
        # the device forms (x - mean) / std in float32 before rounding
        x32 = (np.asarray(X, np.float32) - np.asarray(mean, np.float32)) / np.asarray(std, np.float32)
        return bf16_round(x32)
    return (np.asarray(X, np.float64) - np.asarray(mean, np.float64)) / np.asarray(std, np.float64)


def forward(params, mean, std, X, bf16=True):
    """Returns y (n,) and the activations (x, h1, h2) used by loss_grad."""
    p = bf16_round(params) if bf16 else np.asarray(params, np.float64)
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = _standardise(X, mean, std, bf16)
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    if bf16:
        h1 = bf16_round(h1)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    if bf16:
        h2 = bf16_round(h2)
    y = h2 @ w3 + b3
    return y, (x, h1, h2, p)


def loss_grad(params, mean, std, X, t, bf16=True):
    """Loss 0.5 mean_i (y_i - t_i)^2 and its gradient (NPARAM,)."""
    y, (x, h1, h2, p) = forward(params, mean, std, X, bf16)
    W1, b1, W2, b2, w3, b3 = unpack(p)
    n = y.shape[0]
    r = y - np.asarray(t, np.float64)
    loss = 0.5 * np.dot(r, r) / n
    dl = r / n                                  # d loss / d y
    g = np.zeros(NPARAM)
    g[OFF_B3] = dl.sum()
    g[OFF_W3:OFF_B3] = h2.T @ dl
    dh2 = np.outer(dl, w3) * (h2 > 0)           # through the second ReLU
    g[OFF_B2:OFF_W3] = dh2.sum(axis=0)
    g[OFF_W2:OFF_B2] = (dh2.T @ h1).ravel()
    dh1 = (dh2 @ W2) * (h1 > 0)                 # through the first ReLU
    g[OFF_B1:OFF_W2] = dh1.sum(axis=0)
    g[:OFF_B1] = (dh1.T @ x).ravel()
    return loss, g


def adam_step(p, g, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def node_features(d, gam, mu, uh, n, s0, s1):
    d, gam, mu, uh = (np.asarray(a, np.float64) for a in (d, gam, mu, uh))
    K = d.shape[0]
    spread = (d[K - 1] + gam[K - 1]) - d[0]
    gaps = list(gam[s0:s1]) + list(mu[s0:min(s1, K - 1)])
    gaps = np.sort(np.maximum(np.asarray(gaps), 1e-300))
    c = gaps.shape[0]
    med = gaps[(c + 1) // 2 - 1]
    dist = spread
    for b in (s0, s1):
        if 0 < b < K:
            dist = min(dist, (d[b] - d[b - 1]) + gam[b])
    return np.array([
        np.log2(s1 - s0),
        np.log10(gaps[0] / spread),
        np.log10(med / spread),
        np.log10(max(dist, 1e-300) / spread),
        np.log10(max(np.sum(uh[s0:s1] ** 2), 1e-300)),
        (n - K) / n,
        np.log2(K),
    ])
