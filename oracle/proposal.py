"""FP64 oracle of the learned insertion-site proposal.

TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's CPU legs, never by the GPU
library).  Plain numpy, written for reading against the definitions below.

The proposal replaces the uniform placement of an inserted ion pair (1/V per ion,
Eq. 4) by a density learned from the method's own trial records; its ratio to the
uniform density enters the acceptance rule so that detailed balance holds, the same way
the bias factors B^ins/B^del enter Eqs. 15-16:

* grid: G^3 cells, G = max(3, floor(L / cell_len)); an atom with 32-bit box fractions
  X belongs to cell floor(X G / 2^32) on each axis;
* features of cell c (96): for species s in (cation, anion, water O) and each of the 27
  cells of c's 3x3x3 neighbourhood, 0.25 x the atom count (81), then 0.1 x the Coulomb
  field at c's centre from the charges of those 27 cells, sum_j q_j d_j / max(|d_j|, 0.5)^3
  with d_j the minimum-image vector from atom j to the centre (3), then 12 zeros;
* MLP 96 -> 64 -> 64 -> 2 with ReLU: h1 = relu(f W1 + b1), h2 = relu(h1 W2 + b2),
  logits = h2 W3 + b3; output 0 scores cation sites, output 1 anion sites;
* q_s = (1 - eps) softmax(logits_s over cells) + eps / G^3, eps = 0.1;
* an inserted ion is placed uniformly inside a cell drawn from q_s, so its density is
  q_s(cell) G^3 / V.  Insertion multiplies the Metropolis ratio of Eq. 6 by
  1 / [(q_c G^3)(q_a G^3)] with q from the start (N-pair) state; deletion multiplies the
  ratio of Eq. 8 by (q_c G^3)(q_a G^3) with q from the end (N-pair) state.
"""
from __future__ import annotations

import numpy as np

NFEAT, HID, NOUT, NSPEC = 96, 64, 2, 3
EPS_MIX = 0.1
TWO32 = 4294967296

# flat weight layout shared by name with the C ABI: W1[96,64], b1[64], W2[64,64], b2[64], W3[64,2], b3[2]
SHAPES = [("W1", (NFEAT, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, NOUT)),
          ("b3", (NOUT,))]
N_WEIGHTS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[k:k + n], np.float64).reshape(shp)
        k += n
    return out


def pack(w):
    return np.concatenate([np.asarray(w[name], np.float64).ravel() for name, _ in SHAPES])


def init_weights(seed):
    rng = np.random.default_rng(seed)
    w = {"W1": rng.normal(0, 1 / np.sqrt(NFEAT), (NFEAT, HID)), "b1": np.zeros(HID),
         "W2": rng.normal(0, 1 / np.sqrt(HID), (HID, HID)), "b2": np.zeros(HID),
         "W3": rng.normal(0, 1 / np.sqrt(HID), (HID, NOUT)), "b3": np.zeros(NOUT)}
    return pack(w)


def grid_size(L, cell_len):
    return max(3, int(np.floor(L / cell_len)))


def fixed(x, L):
    """32-bit box fractions (round to nearest), as the library stores positions"""
    y = np.mod(np.asarray(x, np.float64), L)
    return (np.rint(y / L * TWO32).astype(np.uint64) % TWO32).astype(np.uint64)


def species_of(t):
    return {0: 0, 1: 1, 2: 2}.get(int(t), -1)  # water H does not count


def features(x, types, charges, L, G, exclude=()):
    """[G^3, 96] features of every cell (definition in the module docstring)"""
    x = np.asarray(x, np.float64)
    X = fixed(x, L)
    g = ((X * G) >> 32).astype(np.int64)  # cell index per axis
    ex = set(int(e) for e in exclude)
    F = np.zeros((G, G, G, NFEAT))
    h = L / G
    for a in range(len(x)):
        if a in ex:
            continue
        s = species_of(types[a])
        q = charges[int(types[a])]
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    # atom a lies in neighbour cell (offset -d) of cell c = g_a + d
                    cx, cy, cz = (g[a, 0] + dx) % G, (g[a, 1] + dy) % G, (g[a, 2] + dz) % G
                    nidx = (1 - dx) * 9 + (1 - dy) * 3 + (1 - dz)
                    if s >= 0:
                        F[cx, cy, cz, s * 27 + nidx] += 0.25
                    if q != 0.0:
                        centre = (np.array([cx, cy, cz]) + 0.5) * h
                        d = centre - x[a]
                        d -= L * np.round(d / L)
                        r = max(np.sqrt(d @ d), 0.5)
                        F[cx, cy, cz, 81:84] += 0.1 * q * d / r**3
    return F.reshape(G * G * G, NFEAT)


def bf16(a):
    """round to bfloat16 (nearest, ties to even) through binary32"""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(flat, X, emulate_bf16=False):
    """logits [n, 2] of feature rows X [n, 96] and the activations the backward pass needs;
    emulate_bf16 rounds features, weights and hidden activations to bfloat16 and each
    layer's sum to binary32, the precision in which the GPU kernel evaluates the network
    (and so takes its ReLU and cell decisions)"""
    w = unpack(flat)
    r = bf16 if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    f32 = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if emulate_bf16 else (lambda a: a)
    Xr = r(X)
    z1 = f32(f32(Xr @ r(w["W1"])) + w["b1"])
    h1 = r(np.maximum(z1, 0.0))
    z2 = f32(f32(h1 @ r(w["W2"])) + w["b2"])
    h2 = r(np.maximum(z2, 0.0))
    logits = f32(f32(h2 @ r(w["W3"])) + w["b3"])
    return logits, (Xr, z1, h1, z2, h2, emulate_bf16)


def forward_abs(flat, X):
    """the forward pass on absolute values with every unit active: bounds |logit| and how
    far operand rounding can move each logit"""
    w = unpack(flat)
    a1 = np.abs(X) @ np.abs(w["W1"]) + np.abs(w["b1"])
    a2 = a1 @ np.abs(w["W2"]) + np.abs(w["b2"])
    return a2 @ np.abs(w["W3"]) + np.abs(w["b3"])


def backward(flat, cache, dlogits, absolute=False):
    """gradients of sum(dlogits * logits) with respect to every weight (flat layout);
    absolute=True runs the same products on absolute values, which bounds how far rounding
    of the operands can move each gradient element"""
    w = unpack(flat)
    X, z1, h1, z2, h2, emulate = cache
    r = bf16 if emulate else (lambda v: v)
    a = np.abs if absolute else (lambda v: v)
    g = {}
    g["W3"] = a(h2).T @ a(dlogits)
    g["b3"] = a(dlogits).sum(0)
    dh2 = a(dlogits) @ a(r(w["W3"])).T
    dz2 = dh2 * (z2 > 0)
    g["W2"] = a(h1).T @ dz2
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ a(r(w["W2"])).T
    dz1 = dh1 * (z1 > 0)
    g["W1"] = a(X).T @ dz1
    g["b1"] = dz1.sum(0)
    return pack(g)


def soft_target(y, y0):
    """training target of a record with insertion-direction exponent y: the Metropolis
    acceptance min(1, e^(y - y0)) of the move, shifted by y0 so that the targets of short
    training trajectories are not all vanishingly small (a constant shift moves every
    logit alike and leaves the softmax proposal unchanged in the small-target limit)"""
    return np.exp(np.minimum(np.asarray(y, np.float64) - y0, 0.0))


def bce(logit, t):
    """binary cross-entropy of a logit against a soft target, in the overflow-free form"""
    return np.maximum(logit, 0.0) - logit * t + np.log1p(np.exp(-np.abs(logit)))


def bce_loss_grad(flat, Xc, Xa, tc, ta, absolute=False, emulate_bf16=False):
    """loss = (1/n) sum_records [BCE(cation logit of the cation cell, t_c) +
    BCE(anion logit of the anion cell, t_a)] and its flat gradient"""
    n = len(tc)
    lc, cc = forward(flat, Xc, emulate_bf16)
    la, ca = forward(flat, Xa, emulate_bf16)
    loss = (bce(lc[:, 0], tc).sum() + bce(la[:, 1], ta).sum()) / n
    sig = lambda z: 0.5 * (1.0 + np.tanh(0.5 * z))
    dc = np.zeros_like(lc)
    dc[:, 0] = (sig(lc[:, 0]) - tc) / n
    da = np.zeros_like(la)
    da[:, 1] = (sig(la[:, 1]) - ta) / n
    return loss, backward(flat, cc, dc, absolute) + backward(flat, ca, da, absolute)


def adam_step(flat, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """one Adam update (Kingma and Ba 2015) of the flat weights; step counts from 1"""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1**step)
    vh = v / (1 - b2**step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def proposal_q(logits, eps=EPS_MIX):
    """[N_cell, 2] proposal probabilities over cells"""
    z = logits - logits.max(0)
    p = np.exp(z)
    p /= p.sum(0)
    return (1 - eps) * p + eps / logits.shape[0]
