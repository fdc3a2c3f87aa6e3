"""Learned (l, q) controller around the randomized SVD, float64.

TEST INFRASTRUCTURE ONLY (oracle); nothing in the product path may import it.

The paper has no learned component.  What it fixes, and what this module
restates, is the machinery the controller is wrapped in:

* the probe is a thin Gaussian sketch Y = A G of 16 columns (Sec. 4, Fig. RSVD,
  with l = 16): its singular values are the controller's view of the decay of
  A's spectrum;
* the labels are what the paper's tolerance-driven range finder (Sec. 12.3,
  Fig. greedy_blocked, and the power variant in that figure's caption) needs:
  for each q in {0, 1, 2, 3} the rank l_q at which ||A - Q B||_Fro <= eps;
* the judge of a prediction is the randomized residual estimate of Sec. 13/14:
  E = (A - U D V*) G for a thin Gaussian G, with E||E(:, i)||^2 = ||A - U D
  V*||_Fro^2 (eq. (infomm)) and the spectral bound of Lemma thm:aposteriori.

Network (readings, not fixed by the paper): 17 inputs -> Linear(17, 128) ->
ReLU -> Linear(128, 128) -> ReLU -> Linear(128, 20).  Outputs 0..15 are the
logits of l in {16, 32, ..., 256} (class c <-> l = 16 (c + 1)); outputs
16..19 are the logits of q in {0, 1, 2, 3}.  The loss of one sample with
labels (c*, q*) is

    -log p_l[c*] - log p_q[q*] + lam * sum_{c < c*} p_l[c]

(cross-entropy on both heads plus a penalty on the probability of choosing
too small an l, since a too-small l costs a fallback).  Parameters are kept
in one flat array, in this order: W1 (128 x 17, row-major [out][in]), b1 (128),
W2 (128 x 128), b2 (128), W3 (20 x 128), b3 (20).
"""
import numpy as np

from .philox import gaussian, STREAM_SKETCH, STREAM_CERTIFY
from .adaptive import adaptive_blocked

D_IN = 17
HID = 128
N_L = 16
N_Q = 4
N_OUT = N_L + N_Q
PROBE = 16
FEAT_FLOOR = -3.0
Q_CHOICES = (0, 1, 2, 3)
L_STEP = 16

SHAPES = [("W1", (HID, D_IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (N_OUT, HID)), ("b3", (N_OUT,))]


def n_params():
    return sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    """Views of the flat parameter vector as the six named arrays."""
    theta = np.asarray(theta, dtype=np.float64)
    out, off = {}, 0
    for name, shp in SHAPES:
        size = int(np.prod(shp))
        out[name] = theta[off:off + size].reshape(shp)
        off += size
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


# ------------------------------------------------------------------ probe --
def probe_singular_values(A, seed):
    """Singular values of the probe sketch Y = A G, G = the first 16 columns
    of the Omega stream (so the probe is a prefix of the fixed-rank sketch)."""
    A = np.asarray(A, dtype=np.float64)
    w = min(PROBE, A.shape[1])
    G = gaussian(A.shape[1], w, seed, STREAM_SKETCH)
    s = np.linalg.svd(A @ G, compute_uv=False)
    out = np.zeros(PROBE)
    out[:len(s)] = s
    return out


def features(sig, m, n):
    """Controller input: log10(sigma_i / sigma_1) for i = 2..16, clipped below
    at -3, then log2(m) / 16 and log2(n) / 16.  (The floor is a reading: a
    binary32 probe resolves singular-value ratios only down to about
    sqrt(u32) ~ 2.4e-4, so ratios below 1e-3 carry no reliable information.)"""
    sig = np.asarray(sig, dtype=np.float64)
    f = np.full(D_IN, FEAT_FLOOR)
    if sig[0] > 0:
        r = sig[1:PROBE] / sig[0]
        with np.errstate(divide="ignore"):
            f[:PROBE - 1] = np.maximum(np.log10(np.maximum(r, 0.0)), FEAT_FLOOR)
    f[PROBE - 1] = np.log2(m) / 16.0
    f[PROBE] = np.log2(n) / 16.0
    return f


def probe_features(A, seed):
    A = np.asarray(A)
    return features(probe_singular_values(A, seed), A.shape[0], A.shape[1])


# -------------------------------------------------------------------- MLP --
def forward(theta, X):
    """Logits (N x 20) and the hidden activations."""
    P = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    H1 = np.maximum(X @ P["W1"].T + P["b1"], 0.0)
    H2 = np.maximum(H1 @ P["W2"].T + P["b2"], 0.0)
    Z = H2 @ P["W3"].T + P["b3"]
    return Z, H1, H2


def softmax(z):
    z = z - z.max(axis=-1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=-1, keepdims=True)


def loss_and_grad(theta, X, yl, yq, lam):
    """Mean loss over the batch and its gradient with respect to theta."""
    P = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    yl = np.asarray(yl, dtype=np.int64)
    yq = np.asarray(yq, dtype=np.int64)
    N = X.shape[0]
    Z, H1, H2 = forward(theta, X)
    pl = softmax(Z[:, :N_L])
    pq = softmax(Z[:, N_L:])
    rows = np.arange(N)
    below = np.arange(N_L)[None, :] < yl[:, None]          # c < c*
    under = np.sum(pl * below, axis=1)                      # P(l too small)
    loss = np.mean(-np.log(pl[rows, yl]) - np.log(pq[rows, yq]) + lam * under)
    # d loss / d logits
    dZl = pl.copy()
    dZl[rows, yl] -= 1.0
    dZl += lam * pl * (below - under[:, None])
    dZq = pq.copy()
    dZq[rows, yq] -= 1.0
    dZ = np.concatenate([dZl, dZq], axis=1) / N
    g = {}
    g["W3"] = dZ.T @ H2
    g["b3"] = dZ.sum(axis=0)
    dH2 = (dZ @ P["W3"]) * (H2 > 0)
    g["W2"] = dH2.T @ H1
    g["b2"] = dH2.sum(axis=0)
    dH1 = (dH2 @ P["W2"]) * (H1 > 0)
    g["W1"] = dH1.T @ X
    g["b1"] = dH1.sum(axis=0)
    return float(loss), pack(g)


def adam_step(theta, grad, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, ICLR 2015, Algorithm 1), step t >= 1.
    Returns the new (theta, m1, m2)."""
    m1 = beta1 * m1 + (1.0 - beta1) * grad
    m2 = beta2 * m2 + (1.0 - beta2) * grad * grad
    mh = m1 / (1.0 - beta1 ** t)
    vh = m2 / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m1, m2


def decide(logits, theta_q=0.9):
    """Prediction from one row of logits: q = argmax of the q head (lowest on
    ties); l class = the smallest c whose cumulative probability reaches
    theta_q (a conservative quantile, since under-predicting costs a
    fallback).  Returns (l, q)."""
    z = np.asarray(logits, dtype=np.float64)
    pl = softmax(z[:N_L])
    q = int(np.argmax(z[N_L:]))
    cum = np.cumsum(pl)
    c = int(np.searchsorted(cum, theta_q - 1e-12))
    c = min(c, N_L - 1)
    return L_STEP * (c + 1), q


# ----------------------------------------------------------------- labels --
def label_from_ranks(ranks, converged, R=256):
    """Label (l class, q) from the adaptive ranks l_q and convergence flags:
    q* minimizes the sketch cost (2q + 2) l_q among the q that met the
    tolerance, ties to the smaller q; l* = l_q*.  If no q met it, the label
    is the largest class with q = 2."""
    best = None
    for q, (r, ok) in enumerate(zip(ranks, converged)):
        if not ok:
            continue
        cost = (2 * q + 2) * r
        if best is None or cost < best[0]:
            best = (cost, q, r)
    if best is None:
        return N_L - 1, 2
    _, q, r = best
    c = min(max((r + L_STEP - 1) // L_STEP - 1, 0), N_L - 1)
    return c, q


def adaptive_ranks(A, tol, seed, b=16, R=256):
    """l_q of the blocked adaptive range finder (Fig. greedy_blocked, power
    variant of its caption) for q in {0, 1, 2, 3}."""
    ranks, conv = [], []
    for q in Q_CHOICES:
        out = adaptive_blocked(A, tol, b=b, seed=seed, q=q, max_rank=R)
        ranks.append(out["rank"])
        conv.append(bool(out["converged"]))
    return ranks, conv


# ------------------------------------------------------------------ judge --
def residual_estimate(A, U, D, V, seed, r=16):
    """E = (A - U D V*) G, G = r columns of the certificate stream.  Returns
    (Frobenius estimate sqrt(mean_i ||E(:, i)||^2) (eq. (infomm)),
    spectral bound 10 sqrt(2/pi) max_i ||E(:, i)|| (Lemma thm:aposteriori
    with alpha = 1/10), column norms)."""
    A = np.asarray(A, dtype=np.float64)
    G = gaussian(A.shape[1], r, seed, STREAM_CERTIFY)
    E = A @ G - U @ (D[:, None] * (V.T @ G))
    cn = np.linalg.norm(E, axis=0)
    return float(np.sqrt(np.mean(cn * cn))), 10.0 * np.sqrt(2.0 / np.pi) * float(cn.max()), cn
