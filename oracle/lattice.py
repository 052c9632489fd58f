"""Lattice constants, restated from the paper (oracle side).

* D3Q19 velocities: the columns of the matrix M in Sec. 2.1, in that order,
  with the rest vector last (index 18).
* D3Q19 weights: Eq. d3q19_weight_function (1/3, 1/18, 1/36 for |c|^2 = 0, 1, 2),
  lattice speed of sound c_s^2 = 1/3 (Sec. 2.1).
* Solid-normal stencil: the 92 vectors with |e|^2 in {1,2,3,4,5,6,8} and the
  eighth-order weights of Eq. eigth_order_weight_function (Sec. 2.2).
* D3Q7 for the dissolved reactant: not in the paper (the paper's reactant is
  the liquid component itself).  Velocities are the first six D3Q19 vectors
  plus rest, weights 1/8 and 1/4, c_s^2 = 1/4.
"""
import itertools

import numpy as np

# --- D3Q19, Sec. 2.1 (columns of M) ----------------------------------------
C19 = np.array(
    [
        [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
        [1, 1, 0], [1, -1, 0], [1, 0, 1], [1, 0, -1], [-1, 1, 0], [-1, -1, 0],
        [-1, 0, 1], [-1, 0, -1], [0, 1, 1], [0, 1, -1], [0, -1, 1], [0, -1, -1],
        [0, 0, 0],
    ],
    dtype=np.int64,
)
Q19 = 19
CS2 = 1.0 / 3.0


def _w19(c2):
    # Eq. d3q19_weight_function
    return {0: 1.0 / 3.0, 1: 1.0 / 18.0, 2: 1.0 / 36.0}[int(c2)]


W19 = np.array([_w19((c * c).sum()) for c in C19])
# opposite direction index: c_opp(i) = -c_i
OPP19 = np.array([int(np.where((C19 == -c).all(axis=1))[0][0]) for c in C19])
# |c_i| (0 for the rest vector), used by the recolouring operator
NORM19 = np.sqrt((C19 * C19).sum(axis=1).astype(np.float64))

# --- D3Q7 for the advection-diffusion populations (ours) -------------------
C7 = np.array(
    [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [0, 0, 0]],
    dtype=np.int64,
)
Q7 = 7
W7 = np.array([1 / 8, 1 / 8, 1 / 8, 1 / 8, 1 / 8, 1 / 8, 1 / 4])
CS2_7 = 1.0 / 4.0
OPP7 = np.array([1, 0, 3, 2, 5, 4, 6])

# --- eighth-order isotropic stencil for the solid normal (Sec. 2.2) ---------
_OMEGA8 = {1: 4 / 45, 2: 1 / 21, 3: 2 / 105, 4: 5 / 504, 5: 1 / 315, 6: 1 / 630, 8: 1 / 5040}
E92 = np.array(
    [
        e
        for e in itertools.product((-2, -1, 0, 1, 2), repeat=3)
        if int(np.dot(e, e)) in _OMEGA8
    ],
    dtype=np.int64,
)
OMEGA92 = np.array([_OMEGA8[int(np.dot(e, e))] for e in E92])

# nearest neighbours (|c|^2 = 1) used by NN(x), Eq. nearest_solid_neighbors
NEAREST6 = [i for i in range(Q19) if (C19[i] * C19[i]).sum() == 1]

# numeric thresholds shared by both precisions (documented readings)
GRAD_EPS = 1e-5      # |grad rho^N| below this: n = 0, H = 0 (above the FP32 noise floor)
SIN2_EPS = 1e-6      # 1 - (n_s . n)^2 below this: wetting leaves n unchanged

# Python-native copies, so that arithmetic with float32 arrays stays float32
# (NumPy scalars would promote it to float64).
C19L = [tuple(int(v) for v in c) for c in C19]
W19L = [float(w) for w in W19]
NORM19L = [float(v) for v in NORM19]
C7L = [tuple(int(v) for v in c) for c in C7]
W7L = [float(w) for w in W7]
E92L = [tuple(int(v) for v in e) for e in E92]
OMEGA92L = [float(w) for w in OMEGA92]
