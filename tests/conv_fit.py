"""Order of convergence from errors at successive resolutions (test helper).

The local slope log2(e(N)/e(2N)) of a second-order scheme tends to 2 as N
grows, but on coarse meshes a higher-order error term can move it away from 2.
leading_order() fits e(N) = A N^-p + B N^-(p+1), the leading term plus one
higher-order correction, to the errors (relative residuals, least squares:
linear in A and B for each p, p scanned on a 1e-3 grid) and returns the
leading exponent p, the order the scheme converges at as N grows.  Fits in
which the two terms nearly cancel are not accepted: A > 0 and, at the finest
resolution, the correction is at most half the leading term
(|B| <= A N_max / 2), i.e. the finest mesh lies in the asymptotic range.
"""
import numpy as np


def local_slopes(N, e):
    N, e = np.asarray(N, float), np.asarray(e, float)
    return np.log(e[:-1] / e[1:]) / np.log(N[1:] / N[:-1])


def leading_order(N, e, lo=0.5, hi=4.0):
    N, e = np.asarray(N, float), np.asarray(e, float)
    best_c, best_p = np.inf, None
    for p in np.arange(lo, hi, 1e-3):
        M = np.stack([N ** -p / e, N ** -(p + 1) / e], axis=1)
        (A, B), *_ = np.linalg.lstsq(M, np.ones_like(e), rcond=None)
        if not (A > 0 and abs(B) <= 0.5 * A * N.max()):
            continue
        r = M @ np.array([A, B]) - 1.0
        c = float(r @ r)
        if c < best_c:
            best_c, best_p = c, float(p)
    return best_p
