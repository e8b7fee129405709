"""16-bit storage of the forward wavefield read by the gradient (oracle, FP64).

The imaging condition of Eq. 3 reads the stored forward wavefield u^j.  The
library may keep every stored level in 16 bits.  This module restates the
storage format as the library's public header defines it, so that the oracle
gradient can be evaluated on exactly the values that the 16-bit forms read:

  * a level on the computational grid is cut, plane by plane, into slabs of 64
    points along x by 2 points along axis 1 (axis 1 is y in 3D and depth in 2D;
    slab (sx, sy) covers x in [64 sx, 64 sx + 64) and axis 1 in [2 sy, 2 sy + 2),
    cut off at the grid's end);
  * each slab has the power-of-two scale s = 2^(floor(log2 amax) - 14), with
    amax the largest |u| in the slab, so that amax / s lies in [2^14, 2^15);
    an all-zero slab has s = 1;
  * each value is kept as u / s rounded to the nearest value of the 16-bit
    format (ties to even): BF16 has 8 significand bits and the exponent range of
    FP32, FP16 has 11 significand bits and is subnormal below 2^-14;
  * the value read back is the stored value times s.

Rounding is written from that definition with FP64 arithmetic (frexp for the
binade, division by a power of two, NumPy's round-half-to-even).  It does not
model the library's own arithmetic: the library rounds its FP32 values, the
oracle its FP64 values.

Test infrastructure only (see the package docstring).
"""

import numpy as np

SLAB_X = 64
SLAB_Y = 2

# significand bits (implicit bit included) and smallest normal exponent
FORMATS = {"bf16": (8, -126), "fp16": (11, -14)}


def round_to_format(x, fmt):
    """x rounded to the nearest value of the 16-bit format (ties to even),
    as float64.  Values must lie inside the format's finite range."""
    p, emin = FORMATS[fmt]
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)                    # |x| = f 2^e, f in [0.5, 1): binade exponent e - 1
    e = np.maximum(e - 1, emin)           # below the normal range the quantum stays at 2^(emin - p + 1)
    quantum = np.ldexp(1.0, e - (p - 1))
    return np.round(x / quantum) * quantum


def slab_scales(level):
    """Per-slab scales of one stored level in array layout ([nz][ny][nx] in 3D,
    [nz][nx] in 2D, where the depth axis is axis 1 of the slabs); returns an
    array [planes][slabs along axis 1][slabs along x]."""
    u = np.asarray(level, dtype=np.float64)
    planes = u.reshape((-1,) + u.shape[-2:])        # 2D: one plane
    n1, nx = planes.shape[1:]
    s1, sx = -(-n1 // SLAB_Y), -(-nx // SLAB_X)
    padded = np.zeros((planes.shape[0], s1 * SLAB_Y, sx * SLAB_X))
    padded[:, :n1, :nx] = np.abs(planes)
    amax = padded.reshape(planes.shape[0], s1, SLAB_Y, sx, SLAB_X).max(axis=(2, 4))
    _, e = np.frexp(amax)                           # amax in [2^(e-1), 2^e)
    return np.where(amax > 0.0, np.ldexp(1.0, e - 1 - 14), 1.0)


def round_level(level, fmt):
    """The values the library reads back for one level stored in `fmt`."""
    u = np.asarray(level, dtype=np.float64)
    planes = u.reshape((-1,) + u.shape[-2:])
    n1, nx = planes.shape[1:]
    s = slab_scales(u)
    s_pt = np.repeat(np.repeat(s, SLAB_Y, axis=1), SLAB_X, axis=2)[:, :n1, :nx]
    return (round_to_format(planes / s_pt, fmt) * s_pt).reshape(u.shape)
