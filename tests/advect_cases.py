"""A MacCormack case where the clamp acts, with its expected pieces computed
from the definitions (shared by the oracle pin and the GPU parity test)."""
import numpy as np


def clamp_case(N=32):
    """A smooth ramp with one spike on the 32^3 box grid, a uniform fractional
    velocity of d = (0.7, -0.35, 1.3) cells per step (RK3 of a uniform field is
    the straight backtrace x - d), and the MacCormack correction's pieces
    computed here from their definitions on a dense array: trilinear samples
    over the 8 named cell centres, q_hat(x) = q(x - d), q_tilde(x) =
    q_hat(x + d), r = q_hat + (q - q_tilde) / 2."""
    dtime = 0.01
    d = np.array([0.7, -0.35, 1.3])
    dense = np.zeros((N, N, N))
    r = np.arange(4, 28)
    I, J, K = np.meshgrid(r, r, r, indexing="ij")
    dense[I, J, K] = 0.05 * (I + 2 * J - K) / N
    dense[16, 15, 17] += 1.0                                  # the spike

    def window(field, p):
        X = p - 0.5
        b = np.floor(X).astype(np.int64)
        f = X - b
        s = np.zeros(p.shape[:-1])
        vals = []
        for a in (0, 1):
            for c in (0, 1):
                for e in (0, 1):
                    v = field[b[..., 0] + a, b[..., 1] + c, b[..., 2] + e]
                    w = ((f[..., 0] if a else 1 - f[..., 0]) * (f[..., 1] if c else 1 - f[..., 1])
                         * (f[..., 2] if e else 1 - f[..., 2]))
                    s = s + w * v
                    vals.append(v)
        vals = np.stack(vals, -1)
        return s, vals.min(-1), vals.max(-1)

    q = 10
    ri = np.arange(q, N - q)
    x = np.stack(np.meshgrid(ri, ri, ri, indexing="ij"), -1).astype(np.float64) + 0.5
    xe = np.stack(np.meshgrid(np.arange(6, N - 6), np.arange(6, N - 6), np.arange(6, N - 6), indexing="ij"), -1) + 0.5
    qhat_e, _, _ = window(dense, xe - d)                     # q_hat on a wider block, for q_tilde's window
    qhat_dense = np.zeros_like(dense)
    qhat_dense[6:N - 6, 6:N - 6, 6:N - 6] = qhat_e
    qhat, lo_f, hi_f = window(dense, x - d)                  # forward sample and its 8 values
    qtil, lo_b, hi_b = window(qhat_dense, x + d)             # backward sample of q_hat
    qx = dense[q:N - q, q:N - q, q:N - q]
    rr = qhat + 0.5 * (qx - qtil)
    _, lo_s, hi_s = window(dense, x)                         # the voxel's own 8 cells
    _, lo_bq, hi_bq = window(dense, x + d)                   # q's values around the backward sample
    return dtime, d, dense, q, rr, (lo_f, hi_f), (lo_s, hi_s), (lo_bq, hi_bq)
