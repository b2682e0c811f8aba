"""Plain FP64 reference of the learned coarse-grid correction (not in the paper).

TEST INFRASTRUCTURE ONLY (tests, smoke, benchmark baselines).

The correction is a per-node multilayer perceptron applied to a coarse
Hermite-leapfrog solution:

    features f(J) of coarse primal node J (2D, m = 3, 16 slots per field):
      - p at the 3x3 primal nodes J + {-1, 0, 1}^2            (9 x 16 = 144)
      - u and v at the 4 dual vertices of J's cell
        (dual nodes J + {-1, 0}^2, the p-half stencil)         (4 x 32 = 128)
      - the time feature t (one value)                         (1)
      zero-padded to N_IN = 288 inputs, all multiplied by feat_scale except t;
    y = relu(relu(f W1 + b1) W2 + b2) W3 + b3      (288 -> 128 -> 128 -> 16)
    p~(J) += out_scale * y                          (16 slot corrections)

Training minimises the mean over rows and outputs of (y - target)^2, with
target = (restricted fine p - coarse p) / out_scale.  The restriction of a
fine grid (ratio r nodes per coarse cell) to the coarse primal nodes J takes
fine primal node r*J and rescales slot a by r^{|a|} (scaled derivatives carry
h^{|a|}/a!, and h_coarse = r h_fine).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 288, 128, 16


def init_params(rng, n_in=N_IN, n_h=N_H, n_out=N_OUT):
    """He-style initial weights (float64)."""
    return {
        "W1": rng.standard_normal((n_in, n_h)) * np.sqrt(2.0 / n_in), "b1": np.zeros(n_h),
        "W2": rng.standard_normal((n_h, n_h)) * np.sqrt(2.0 / n_h), "b2": np.zeros(n_h),
        "W3": rng.standard_normal((n_h, n_out)) * np.sqrt(1.0 / n_h), "b3": np.zeros(n_out),
    }


def _identity(a):
    return a


def forward(params, X, operand_round=None):
    """Returns (Y, cache) with the pre-activations needed by backward.

    operand_round (optional) is applied to both operands of every matrix product (not to
    the bias additions): the precision in which the network's tensor-core products see
    their inputs (BF16 for the learned correction), the sums themselves exact."""
    r = operand_round or _identity
    Z1 = r(X) @ r(params["W1"]) + params["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = r(H1) @ r(params["W2"]) + params["b2"]
    H2 = np.maximum(Z2, 0.0)
    Y = r(H2) @ r(params["W3"]) + params["b3"]
    return Y, (X, Z1, H1, Z2, H2)


def loss_and_grads(params, X, T, operand_round=None):
    """Mean squared error over all rows and outputs and its gradients by back-propagation
    (exact when operand_round is None; otherwise every product's operands are rounded as
    in forward, the back-propagation the tensor cores carry out)."""
    r = operand_round or _identity
    Y, (X, Z1, H1, Z2, H2) = forward(params, X, operand_round)
    n = Y.size
    R = Y - T
    loss = float(np.sum(R * R) / n)
    dY = 2.0 * R / n
    g = {"W3": r(H2).T @ r(dY), "b3": dY.sum(axis=0)}
    dH2 = (r(dY) @ r(params["W3"]).T) * (Z2 > 0)
    g["W2"] = r(H1).T @ r(dH2)
    g["b2"] = dH2.sum(axis=0)
    dH1 = (r(dH2) @ r(params["W2"]).T) * (Z1 > 0)
    g["W1"] = r(X).T @ r(dH1)
    g["b1"] = dH1.sum(axis=0)
    return loss, g


def restrict_p(p_fine, n_fine, ratio, m=3):
    """Fine p (host layout, 2D) at the coarse primal nodes, slot a scaled by ratio^{|a|}."""
    nf0, nf1 = n_fine
    nq = (m + 1) ** 2
    pf = np.asarray(p_fine).reshape(nf1, nf0, nq)
    pc = pf[::ratio, ::ratio, :].copy()
    for q in range(nq):
        a0, a1 = q % (m + 1), q // (m + 1)
        pc[:, :, q] *= float(ratio) ** (a0 + a1)
    return pc.reshape(-1, nq)


def features(p, u, ncell, nodes, feat_scale, t_feature, m=3):
    """Feature rows (len(nodes), N_IN) of the listed coarse primal nodes (host layout input)."""
    n0, n1 = ncell
    nq = (m + 1) ** 2
    P = np.asarray(p).reshape(n1, n0, nq)
    U = np.asarray(u).reshape(2, n1, n0, nq)
    out = np.zeros((len(nodes), N_IN))
    for r, node in enumerate(nodes):
        jx, jy = node % n0, node // n0
        col = 0
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                out[r, col:col + nq] = feat_scale * P[(jy + dy) % n1, (jx + dx) % n0]
                col += nq
        for comp in range(2):
            for vy in (-1, 0):
                for vx in (-1, 0):
                    out[r, col:col + nq] = feat_scale * U[comp, (jy + vy) % n1, (jx + vx) % n0]
                    col += nq
        out[r, col] = t_feature
    return out


def adam_step(params, grads, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015, Algorithm 1), in float64, in place on params,
    m1 and m2 (dicts of arrays keyed like params); t is the 1-based step count.

    First and second raw moments are exponential averages of g and g*g; each is divided
    by its bias (1 - beta^t) before the step lr * m1_hat / (sqrt(m2_hat) + eps)."""
    for k in params:
        g = grads[k]
        m1[k] = beta1 * m1[k] + (1.0 - beta1) * g
        m2[k] = beta2 * m2[k] + (1.0 - beta2) * g * g
        m1_hat = m1[k] / (1.0 - beta1 ** t)
        m2_hat = m2[k] / (1.0 - beta2 ** t)
        params[k] = params[k] - lr * m1_hat / (np.sqrt(m2_hat) + eps)
