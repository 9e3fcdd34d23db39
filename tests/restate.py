"""Independent restatements of the random draws, written from their published definitions,
for pins that recompute an oracle result from first principles.

None of this calls the oracle or the library:
- Philox4x64-10 comes from numpy's own implementation (numpy advances its 256-bit counter
  once before producing a block, so the block of counter c comes from a generator started
  at c - 1);
- U53(w) = (w >> 11) 2^-53, exact in FP64;
- Box-Muller (Box and Muller, 1958): u1 = 1 - U53(w0) in (0, 1], u2 = U53(w1),
  g0 = sqrt(-2 ln u1) cos(2 pi u2), g1 = sqrt(-2 ln u1) sin(2 pi u2);
- the grid shift s_d = (U53(w_d) - 1/2) a from counter (t, 0, SHIFT, 0), its z part folded
  into [0, a) when the box has walls (reading R4);
- the rotation axis from counter (t, cell, AXIS, 0): z = 2 U53(w0) - 1, phi = 2 pi U53(w1),
  uniform on the sphere by Archimedes' hat-box theorem (reading R9).
"""
import math

import numpy as np

TAG_INIT, TAG_SHIFT, TAG_AXIS, TAG_THERMO, TAG_WALL = 0, 1, 2, 3, 4


def philox(ctr, key):
    c = 0
    for i, w in enumerate(ctr):
        c |= int(w) << (64 * i)
    c = (c - 1) % (1 << 256)
    start = np.array([(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=start)
    return [int(x) for x in bg.random_raw(4)]


def u53(w):
    return float(int(w) >> 11) * 2.0 ** -53


def box_muller(w0, w1):
    u1 = 1.0 - u53(w0)
    u2 = u53(w1)
    rad = math.sqrt(-2.0 * math.log(u1))
    return rad * math.cos(2.0 * math.pi * u2), rad * math.sin(2.0 * math.pi * u2)


def draw(seed, c0, c1, tag):
    return philox([c0, c1, tag, 0], [seed, 0])


def shift(seed, t, a=1.0, walls_z=False):
    w = draw(seed, t, 0, TAG_SHIFT)
    s = np.array([(u53(w[d]) - 0.5) * a for d in range(3)])
    if walls_z and s[2] < 0.0:
        s[2] += a
    return s


def axis(seed, t, cell):
    w = draw(seed, t, cell, TAG_AXIS)
    z = 2.0 * u53(w[0]) - 1.0
    phi = 2.0 * math.pi * u53(w[1])
    rho = math.sqrt((1.0 - z) * (1.0 + z))
    return np.array([rho * math.cos(phi), rho * math.sin(phi), z])
