"""FP64 oracle of the learned global proposal (test infrastructure; see the
package docstring for who may import it).

The paper has no learned component; this follows the published method of
variational autoregressive networks (D. Wu, L. Wang, P. Zhang, Phys. Rev. Lett.
122 (2019) 080602) used as an independence proposal corrected by a
Metropolis-Hastings step, so the stationary distribution stays the Boltzmann
distribution of Eq. (1) whatever the network has learned.

Network (raster order k = y L + x, zero padding -- an autoregressive mask is
not compatible with periodic padding):
  layer 1 : 5x5 convolution, 1 -> C channels, mask A (taps strictly before the
            centre: dy < 0, or dy = 0 and dx < 0), bias, ReLU;
  layers 2..D-1 : 5x5, C -> C, mask B (mask A plus the centre), bias, ReLU;
  layer D : 5x5, C -> 1, mask B, bias -> logit f_k.
p(s_k = +1 | s_<k) = sigmoid(f_k); log q(s) = sum_k log sigmoid(s_k f_k).
Parameters are (W, b) per layer with W[c_out, c_in, 5, 5] (masked taps unused).
Convolution is correlation: out[y, x] = sum_{dy,dx} W[., ., dy+2, dx+2] in[y+dy, x+dx].

Precision: FP64 throughout by default.  The task fixes BF16 weights and
activations for this network; with ``act="bf16"`` every stored activation
(the output of each ReLU) is rounded to BF16 (round to nearest, ties to even),
so the oracle computes the same function as a BF16 implementation -- all
arithmetic stays FP64.
"""
from __future__ import annotations

import numpy as np

K = 5
R = K // 2


def taps(mask: str):
    """(dy, dx) offsets of a mask, in raster order."""
    out = []
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            if dy < 0 or (dy == 0 and (dx < 0 or (mask == "B" and dx == 0))):
                out.append((dy, dx))
    return out


def shift(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """y[..., i, j] = x[..., i + dy, j + dx], zero outside the lattice."""
    out = np.zeros_like(x)
    H, W = x.shape[-2:]
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    out[..., ys:ye, xs:xe] = x[..., ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def round_bf16(x) -> np.ndarray:
    """Round to the nearest BF16 value (8-bit significand), ties to even, via
    the FP32 bit pattern: add 0x7FFF plus the lowest kept bit, clear the low
    16 bits."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(depth: int = 6, channels: int = 32, seed: int = 0, scale: float = 1.0):
    rng = np.random.default_rng(seed)
    params = []
    for l in range(depth):
        cin = 1 if l == 0 else channels
        cout = 1 if l == depth - 1 else channels
        ntap = len(taps("A" if l == 0 else "B"))
        std = scale * np.sqrt(2.0 / (cin * ntap))
        W = rng.normal(0.0, std, size=(cout, cin, K, K))
        b = np.zeros(cout)
        params.append((W, b))
    return params


def masked(params):
    """Zero the taps outside each layer's mask."""
    out = []
    for l, (W, b) in enumerate(params):
        m = np.zeros((K, K))
        for dy, dx in taps("A" if l == 0 else "B"):
            m[dy + R, dx + R] = 1.0
        out.append((W * m, b))
    return out


def forward(params, s: np.ndarray, act: str = "fp64"):
    """s: (B, L, L) of +-1.  Returns logits f (B, L, L) and the per-layer cache
    [(input, pre-activation)] for the backward pass; act="bf16" rounds each
    ReLU output to BF16."""
    x = s[:, None, :, :].astype(np.float64)
    cache = []
    D = len(params)
    for l, (W, b) in enumerate(params):
        mask = "A" if l == 0 else "B"
        z = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:])
        for dy, dx in taps(mask):
            xs = shift(x, dy, dx)  # (B, cin, L, L)
            z += np.einsum("oi,bixy->boxy", W[:, :, dy + R, dx + R], xs)
        z += b[None, :, None, None]
        cache.append((x, z))
        x = np.maximum(z, 0.0) if l < D - 1 else z
        if act == "bf16" and l < D - 1:
            x = round_bf16(x)
    return x[:, 0], cache


def log_sigmoid(t):
    return -np.logaddexp(0.0, -t)


def log_prob(params, s: np.ndarray, act: str = "fp64") -> np.ndarray:
    """log q(s) per configuration (FP64 accumulation)."""
    f, _ = forward(params, s, act)
    return log_sigmoid(s * f).reshape(len(s), -1).sum(axis=1)


def log_prob_sym(params, s: np.ndarray, act: str = "fp64") -> np.ndarray:
    """log q_sym(s), q_sym(s) = (q(s) + q(-s)) / 2 (symmetry under the global
    spin flip, Wu-Wang-Zhang)."""
    return np.logaddexp(log_prob(params, s, act), log_prob(params, -s, act)) - np.log(2.0)


def _backward(params, cache, masks, grad_f, mode: str = "grad"):
    """Backward pass from d loss / d f (grad_f, (B, L, L)) through the layers.
    masks[l] (l < D - 1): the ReLU derivative of layer l's output (1 where the
    output is positive).  mode "grad": the gradient; "scale": per element the
    sum of |terms| through the whole pass (|grad_f| in, |W| in the products);
    "direct": per element the sum of |terms| of its own last contraction only,
    |upstream gradient| x |activation| with the true upstream gradient.
    Returns [(dW, db)] per layer."""
    D = len(params)
    grad_out = (np.abs(grad_f) if mode == "scale" else grad_f)[:, None, :, :]
    out = [None] * D
    for l in range(D - 1, -1, -1):
        W, b = params[l]
        x, _ = cache[l]
        dz = grad_out if l == D - 1 else grad_out * masks[l]
        mask = "A" if l == 0 else "B"
        dW = np.zeros_like(W)
        dx_in = np.zeros_like(x)
        Wb = np.abs(W) if mode == "scale" else W
        for dy, dx in taps(mask):
            xs = shift(x, dy, dx)
            if mode == "grad":
                dW[:, :, dy + R, dx + R] = np.einsum("boxy,bixy->oi", dz, xs)
            elif mode == "scale":
                dW[:, :, dy + R, dx + R] = np.einsum("boxy,bixy->oi", dz, np.abs(xs))
            else:
                dW[:, :, dy + R, dx + R] = np.einsum("boxy,bixy->oi", np.abs(dz), np.abs(xs))
            # x enters z at (y, x) via x[y+dy, x+dx]: scatter back with the opposite shift
            dx_in += shift(np.einsum("oi,boxy->bixy", Wb[:, :, dy + R, dx + R], dz), -dy, -dx)
        out[l] = (dW, (np.abs(dz) if mode == "direct" else dz).sum(axis=(0, 2, 3)))
        grad_out = dx_in
    return out


def _grad_f(s, f):
    """d loss / d f of loss = -mean_b log q(s_b): -(1/B) s sigmoid(-s f)."""
    return -(s * np.exp(-np.logaddexp(0.0, s * f))) / len(s)


def loss_and_grad(params, s: np.ndarray, act: str = "fp64"):
    """Negative mean log-likelihood -mean_b log q(s_b) and its gradient (of
    the network with act-rounded activations, the rounding treated as part of
    the function as a BF16 implementation does)."""
    B = len(s)
    f, cache = forward(params, s, act)
    loss = -log_sigmoid(s * f).reshape(B, -1).sum(axis=1).mean()
    masks = [(z > 0).astype(np.float64) for _, z in cache[:-1]]
    return float(loss), _backward(params, cache, masks, _grad_f(s, f))


def grad_scale(params, s: np.ndarray, act: str = "fp64", propagate: bool = True):
    """Per parameter, a magnitude scale of its gradient sum.
    propagate=True: the sum of the absolute values of the terms that make up
    the gradient through the whole backward pass -- the backward of
    loss_and_grad with |dloss/df| at the output, |W| in the products and the
    ReLU masks kept.  If every term an implementation sums carries a relative
    error of at most e, its gradient element errs by at most about e times
    this scale, whatever cancellation happens inside the sums (triangle
    inequality).  propagate=False: only the last contraction in absolute
    values, sum over samples and positions of |upstream gradient| x
    |activation| with the true (signed) upstream gradient -- the scale of the
    element's own sum.  Same structure as grads of loss_and_grad."""
    f, cache = forward(params, s, act)
    masks = [(z > 0).astype(np.float64) for _, z in cache[:-1]]
    return _backward(params, cache, masks, _grad_f(s, f), "scale" if propagate else "direct")


def forward_following(params, s: np.ndarray, acts, eps_rel: float = 2.0 ** -19):
    """Forward pass with BF16 activations (as act="bf16") that checks another
    implementation's hidden activations acts[l] ((B, L, L, C), layer l =
    0 .. D - 2, after the ReLU) element by element, and adopts the other value
    where -- and only where -- this FP64 run's own pre-activation z lies within
    eps_rel * S of a decision boundary of the activation (a BF16 rounding
    midpoint or the ReLU kink), S = sum over the taps of |W| |x| + |b|, the
    scale of an FP32 accumulation's error: there a sum in another precision may
    legitimately land on the other side (the counterpart of the heat-bath's
    near-threshold decisions).  Downstream layers then see the adopted value.
    Returns (f, cache, masks, n_near, n_bad): masks[l] = 1 where the (adopted)
    output of layer l is positive; n_near counts adopted values, n_bad values
    that differ although z is not that close to a boundary."""
    x = s[:, None, :, :].astype(np.float64)
    cache, masks = [], []
    near = bad = 0
    D = len(params)
    for l, (W, b) in enumerate(params):
        mask = "A" if l == 0 else "B"
        z = np.zeros((x.shape[0], W.shape[0]) + x.shape[2:])
        S = np.zeros_like(z)
        for dy, dx in taps(mask):
            xs = shift(x, dy, dx)
            z += np.einsum("oi,bixy->boxy", W[:, :, dy + R, dx + R], xs)
            S += np.einsum("oi,bixy->boxy", np.abs(W[:, :, dy + R, dx + R]), np.abs(xs))
        z += b[None, :, None, None]
        S += np.abs(b)[None, :, None, None]
        cache.append((x, z))
        if l == D - 1:
            x = z
            break
        own = round_bf16(np.maximum(z, 0.0))
        lo = round_bf16(np.maximum(z - eps_rel * S, 0.0))
        hi = round_bf16(np.maximum(z + eps_rel * S, 0.0))
        other = np.transpose(np.asarray(acts[l], dtype=np.float64), (0, 3, 1, 2))
        differ = other != own
        within = (other >= lo) & (other <= hi)
        near += int((differ & within).sum())
        bad += int((differ & ~within).sum())
        x = np.where(differ & within, other, own)
        masks.append((x > 0).astype(np.float64))
    return x[:, 0], cache, masks, near, bad


def loss_and_grad_following(params, s: np.ndarray, acts, eps_rel: float = 2.0 ** -19):
    """loss_and_grad(act="bf16") on the forward pass of forward_following:
    returns (loss, grads, scale, direct, n_near, n_bad) with the two
    magnitude scales of grad_scale (propagated and direct) on the same pass."""
    B = len(s)
    f, cache, masks, near, bad = forward_following(params, s, acts, eps_rel)
    loss = -log_sigmoid(s * f).reshape(B, -1).sum(axis=1).mean()
    g = _grad_f(s, f)
    return (float(loss), _backward(params, cache, masks, g), _backward(params, cache, masks, g, "scale"),
            _backward(params, cache, masks, g, "direct"), near, bad)


def hidden_activations(params, s: np.ndarray):
    """The BF16 hidden activations of act="bf16" as (B, L, L, C) per layer
    0 .. D - 2 (the layout forward_following takes)."""
    _, cache = forward(params, s, "bf16")
    return [np.transpose(x, (0, 2, 3, 1)) for x, _ in cache[1:]]


def sample(params, n: int, L: int, uniforms: np.ndarray, act: str = "fp64") -> np.ndarray:
    """Autoregressive sampling, one position at a time in raster order:
    s_k = +1 iff u_k < sigmoid(f_k(s_<k)).  uniforms: (n, L*L) in (0, 1].
    Slow (L^2 full forward passes): for small lattices only."""
    s = np.zeros((n, L, L))
    for k in range(L * L):
        y, x = divmod(k, L)
        f, _ = forward(params, s, act)
        p = 1.0 / (1.0 + np.exp(-f[:, y, x]))
        s[:, y, x] = np.where(uniforms[:, k] < p, 1.0, -1.0)
    return s


def ising_energy(s: np.ndarray) -> np.ndarray:
    """H of Eq. (1) on the periodic torus, per configuration."""
    return -(s * np.roll(s, -1, axis=-1)).sum(axis=(-2, -1)) - (s * np.roll(s, -1, axis=-2)).sum(axis=(-2, -1))


def mh_accept_logratio(params, beta: float, s_cur: np.ndarray, s_prop: np.ndarray,
                       act: str = "fp64") -> np.ndarray:
    """log of the Metropolis-Hastings ratio for an independence proposal from
    q_sym: -beta (E' - E) + log q_sym(s) - log q_sym(s')."""
    return (-beta * (ising_energy(s_prop) - ising_energy(s_cur)) + log_prob_sym(params, s_cur, act)
            - log_prob_sym(params, s_prop, act))


def conditionals(params, s: np.ndarray, act: str = "fp64") -> np.ndarray:
    """p(s_k = +1 | s_<k) at every position of each configuration, from one
    forward pass: the probability the sampler compared its uniform with at
    position k, given that it had drawn s_<k."""
    f, _ = forward(params, np.asarray(s, dtype=np.float64), act)
    return 1.0 / (1.0 + np.exp(-f))


# Random streams of the proposal, keyed by the network's 64-bit seed (key =
# seed low, seed high), in the counter layout of the Philox stream the local
# sweeps use:
#   sampler : position k of the sample with id i takes word k & 3 of the block
#             (k >> 2, round, TAG_SAMPLE, i);
#   MH step : chain c takes the block (0, round, TAG_MH, c); word 0 gives the
#             accept uniform, the top bit of word 1 the global flip.
# A uniform is ((r >> 8) + 1) 2^-24, in (0, 1].
TAG_SAMPLE = 0x21000000
TAG_MH = 0x22000000


def sampler_uniforms(seed: int, rnd: int, ids, L: int) -> np.ndarray:
    """(len(ids), L*L) uniforms of the sampler's stream."""
    from . import philox_words, uniform01
    return np.stack([uniform01(philox_words(seed, rnd, TAG_SAMPLE, int(i), L * L)) for i in ids])


def mh_draws(seed: int, rnd: int, chain_ids):
    """(accept uniform, global flip) per chain of one MH round."""
    from . import philox_words, uniform01
    w = np.stack([philox_words(seed, rnd, TAG_MH, int(c), 2) for c in chain_ids])
    return uniform01(w[:, 0]), (w[:, 1] >> 31).astype(bool)
