"""Oracle of the learned right preconditioner (a message-passing network over tet-face adjacency).

The paper solves its pressure systems without a preconditioner; this network is the learned
preconditioner of the build's target workload, applied as M(r) ~ A^-1 r inside flexible GMRES.
Plain FP64 numpy with a hand-written backward pass; pinned against finite differences.

Network (hidden width H, L message-passing layers), per tet i with face neighbours N(i):
  s      = RMS of r over all entries;  x_i = [r_i / s, g_i]        (g_i: geometry features)
  h0_i   = relu(We x_i + be)
  m_i    = Sum_{n in N(i)} h_n^{l-1}
  h^l_i  = relu(Ws^l h^{l-1}_i + Wm^l m_i + b^l),   l = 1..L
  M(r)_i = s (Wd h^L_i + bd)
Loss over pairs (r, e) with A e = r:  mean ||M(r) - e||^2 / ||e||^2.
"""
import numpy as np


def init_params(F, C, H=64, L=3, seed=0):
    rng = np.random.default_rng(seed)
    p = {"We": rng.standard_normal((H, F)) * np.sqrt(2.0 / F), "be": np.zeros(H)}
    for l in range(L):
        p[f"Ws{l}"] = rng.standard_normal((H, H)) * np.sqrt(1.0 / H)
        p[f"Wm{l}"] = rng.standard_normal((H, H)) * np.sqrt(0.25 / H)
        p[f"b{l}"] = np.zeros(H)
    p["Wd"] = rng.standard_normal((C, H)) * np.sqrt(1.0 / H) * 0.1
    p["bd"] = np.zeros(C)
    return p


def n_layers(p):
    return sum(1 for k in p if k.startswith("Ws"))


def gather_sum(h, nbr):
    """m_i = Sum over the (up to 4) neighbours of i; nbr (ne, 4) with -1 for none."""
    m = np.zeros_like(h)
    for f in range(nbr.shape[1]):
        ok = nbr[:, f] >= 0
        m[ok] += h[nbr[ok, f]]
    return m


def scatter_sum(g, nbr, ne):
    """Adjoint of gather_sum: d/dh_n of Sum_i <g_i, m_i>."""
    out = np.zeros((ne, g.shape[1]))
    for f in range(nbr.shape[1]):
        ok = nbr[:, f] >= 0
        np.add.at(out, nbr[ok, f], g[ok])
    return out


def forward(p, X, nbr, keep=False):
    L = n_layers(p)
    pre0 = X @ p["We"].T + p["be"]
    h = np.maximum(pre0, 0.0)
    cache = {"X": X, "pre": [pre0], "h": [h], "m": []}
    for l in range(L):
        m = gather_sum(h, nbr)
        pre = h @ p[f"Ws{l}"].T + m @ p[f"Wm{l}"].T + p[f"b{l}"]
        h = np.maximum(pre, 0.0)
        cache["m"].append(m); cache["pre"].append(pre); cache["h"].append(h)
    out = h @ p["Wd"].T + p["bd"]
    return (out, cache) if keep else out


def backward(p, cache, dout, nbr):
    """Gradients of Sum <dout, out> with respect to every parameter."""
    L = n_layers(p)
    ne = dout.shape[0]
    g = {"Wd": dout.T @ cache["h"][L], "bd": dout.sum(0)}
    dh = dout @ p["Wd"]
    for l in reversed(range(L)):
        dpre = dh * (cache["pre"][l + 1] > 0)
        g[f"Ws{l}"] = dpre.T @ cache["h"][l]
        g[f"Wm{l}"] = dpre.T @ cache["m"][l]
        g[f"b{l}"] = dpre.sum(0)
        dh = dpre @ p[f"Ws{l}"] + scatter_sum(dpre @ p[f"Wm{l}"], nbr, ne)
    dpre = dh * (cache["pre"][0] > 0)
    g["We"] = dpre.T @ cache["X"]
    g["be"] = dpre.sum(0)
    return g


def features(r, geom):
    s = np.sqrt(np.mean(r * r))
    s = s if s > 0 else 1.0
    return np.hstack([r / s, geom]), s


def apply(p, r, geom, nbr):
    X, s = features(r, geom)
    return s * forward(p, X, nbr)


def loss_and_grad(p, pairs, geom, nbr):
    """pairs: list of (r, e) with shapes (ne, C).  Returns mean relative squared error and grads."""
    tot = 0.0
    grads = {k: np.zeros_like(v) for k, v in p.items()}
    for r, e in pairs:
        X, s = features(r, geom)
        out, cache = forward(p, X, nbr, keep=True)
        diff = s * out - e
        ee = np.sum(e * e)
        tot += np.sum(diff * diff) / ee
        dout = (2.0 / ee) * diff * s
        for k, v in backward(p, cache, dout, nbr).items():
            grads[k] += v
    n = len(pairs)
    return tot / n, {k: v / n for k, v in grads.items()}


def adam_step(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    t = state.get("t", 0) + 1
    state["t"] = t
    for k in p:
        mk, vk = state.setdefault("m" + k, np.zeros_like(p[k])), state.setdefault("v" + k, np.zeros_like(p[k]))
        mk[:] = b1 * mk + (1 - b1) * g[k]
        vk[:] = b2 * vk + (1 - b2) * g[k] * g[k]
        mh = mk / (1 - b1 ** t)
        vh = vk / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
