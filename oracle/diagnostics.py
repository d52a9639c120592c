"""Divergence and curl diagnostics of an interpolated field, FP64 (test
infrastructure only).

Sec. IV.A ("Divergence and curl"): with the base's magnetisation frozen, the
field it makes inside the slider is sampled at the slider's cell centres for
partial movements x between cells, and judged by

    D(x) = (1/N) sum_i |div H|_i(x),    C(x) = (1/N) sum_i ||curl H||_i(x),

each derivative a two-point central finite difference between the cell's two
neighbours along that axis, (H(i+1) - H(i-1)) / (2 d).  Reading (the paper is
silent on the ends): the sums run over the cells that have both neighbours
along every axis of at least three cells, N counts those cells, and an axis of
fewer than three cells contributes no derivative.
"""

import numpy as np


def div_curl_means(H, cell):
    """(D, C) of a field H (3, nz, ny, nx) in A/m on cells of size cell = (dx, dy, dz) m."""
    H = np.asarray(H, dtype=np.float64)
    _, nz, ny, nx = H.shape
    n = (nx, ny, nz)
    use = [n[a] >= 3 for a in range(3)]
    # interior index ranges per array axis (z, y, x)
    sl = tuple(slice(1, n[a] - 1) if use[a] else slice(0, n[a]) for a in (2, 1, 0))

    def d(c, a):
        """Central difference of component c along axis a on the interior (zero if unused)."""
        if not use[a]:
            return np.zeros(tuple(s.stop - s.start for s in sl))
        ax = 2 - a  # array axis of x, y, z
        lo = list(sl)
        hi = list(sl)
        lo[ax] = slice(sl[ax].start - 1, sl[ax].stop - 1)
        hi[ax] = slice(sl[ax].start + 1, sl[ax].stop + 1)
        return (H[c][tuple(hi)] - H[c][tuple(lo)]) / (2.0 * cell[a])

    div = d(0, 0) + d(1, 1) + d(2, 2)
    curl = np.stack([d(2, 1) - d(1, 2), d(0, 2) - d(2, 0), d(1, 0) - d(0, 1)])
    N = div.size
    if N == 0:
        return 0.0, 0.0
    return float(np.sum(np.abs(div)) / N), float(np.sum(np.sqrt(np.sum(curl * curl, axis=0))) / N)
