"""Reader and fixture-detector builder for tests/golden/split_pixels.txt (test helper)."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "split_pixels.txt")
SPLIT_CODES = {"none": 0, "bbox": 1, "full": 2}
NPT_AZIM = 360  # azimuthal bins of the fixture detector in 2D


def load_fixtures():
    out = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            head, tail = line.split("|")
            tok = head.split()
            pid, split, ndim = tok[0], tok[1], int(tok[2])
            vals = [float(v) for v in tok[3:]]
            corners = [(vals[2 * k], vals[2 * k + 1]) for k in range(4)]
            entries = {}
            for item in tail.split():
                key, w = item.split(":")
                if ndim == 1:
                    entries[(int(key),)] = float(Fraction(w))
                    continue
                rb, cb = key.split(",")
                chis = range(NPT_AZIM) if cb == "*" else (int(cb),)
                for c in chis:
                    entries[(int(rb), c)] = float(Fraction(w))
            out.append(dict(id=pid, split=SPLIT_CODES[split], ndim=ndim, corners=corners,
                            entries=entries))
    return out


def fixture_detector(pixels):
    """1-row detector: pixel 0 sets the radial range [0, 10]; each test pixel sits at an
    even column 2 + 2t, separated by masked spacer pixels so that no two test pixels share
    a corner.  Returns (ny, nx, corner_rad, corner_chi, mask, test_pixel_indices)."""
    n = len(pixels)
    nx = 2 + 2 * n - 1
    rad = np.full((2, nx + 1), 5.0)
    chi = np.full((2, nx + 1), 0.5)
    rad[0, 0], rad[1, 0] = 0.0, 10.0
    mask = np.zeros((1, nx), np.uint8)
    mask[0, 1::2] = 1
    cols = []
    for t, corners in enumerate(pixels):
        j = 2 + 2 * t
        (r0, c0), (r1, c1), (r2, c2), (r3, c3) = corners
        rad[0, j], chi[0, j] = r0, c0
        rad[0, j + 1], chi[0, j + 1] = r1, c1
        rad[1, j + 1], chi[1, j + 1] = r2, c2
        rad[1, j], chi[1, j] = r3, c3
        cols.append(j)
    return 1, nx, rad, chi, mask, cols


def column_entries(indptr, indices, data, pixel, npt_rad, ndim):
    """{bin key: weight} of one pixel's column of a CSR matrix."""
    indptr = np.asarray(indptr)
    rows = np.repeat(np.arange(len(indptr) - 1), np.diff(indptr))
    sel = np.asarray(indices) == pixel
    out = {}
    for r, w in zip(rows[sel], np.asarray(data)[sel]):
        key = (int(r),) if ndim == 1 else (int(r % npt_rad), int(r // npt_rad))
        out[key] = float(w)
    return out
