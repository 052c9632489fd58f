"""Synthetic workloads (sizes, seeds, parameters) of the benchmark and parity tests.

The paper's 256^3 bijel geometry is not available; every workload uses a
seeded Gaussian-random-field mask (``synth.grf_mask``) with the structure
class of the paper's sample (bicontinuous, porosity ~0.5-0.6).  Parameters
not stated for a workload take those of the 32^3 periodic case (tau = 1,
sigma = 0.01, beta = 0.7, D = 0.05, no body force).
"""
from dataclasses import dataclass, field

from . import synth
from .lbm import Params


@dataclass
class Workload:
    name: str
    shape: tuple            # (nz, ny, nx)
    shell_k0: float
    porosity: float
    seed: int
    bc_z: int
    params: Params = field(default_factory=Params)

    def mask(self):
        return synth.grf_mask(self.shape, self.shell_k0, self.porosity, self.seed, periodic_z=self.bc_z == 0)

    @property
    def nodes(self):
        nz, ny, nx = self.shape
        return nx * ny * nz


WORKLOADS = {
    # 32^3 periodic, FP32 GPU vs FP64 oracle, 200 steps
    "periodic32": Workload("periodic32", (32, 32, 32), 4, 0.55, 1, 0,
                           Params(tau=1.0, sigma=0.01, beta=0.7, theta_deg=90.0, accel=(1e-6, 0.0, 0.0),
                                  diffusivity=0.05, k_rate=1e-3, c_init=1.0)),
    # reactive flow-through column 128 x 128 x 256, inlet u = 0.005, c = 1 at z = 0, outlet at z = 255
    "column128x128x256": Workload("column128x128x256", (256, 128, 128), 8, 0.5, 2, 1,
                                  Params(tau=1.0, sigma=0.01, beta=0.7, theta_deg=60.0, k_rate=5e-3,
                                         diffusivity=0.05, u_in=0.005, c_in=1.0, c_init=1.0, rho_out=1.0)),
    # the same column recipe at a quarter of the length: small case of the kernel profiles
    "column128x128x64": Workload("column128x128x64", (64, 128, 128), 8, 0.5, 2, 1,
                                 Params(tau=1.0, sigma=0.01, beta=0.7, theta_deg=60.0, k_rate=5e-3,
                                        diffusivity=0.05, u_in=0.005, c_in=1.0, c_init=1.0, rho_out=1.0)),
    # 256^3 periodic precision workload
    "periodic256": Workload("periodic256", (256, 256, 256), 12, 0.5, 3, 0,
                            Params(tau=1.0, sigma=0.01, beta=0.7, theta_deg=60.0, k_rate=1e-3,
                                   diffusivity=0.05, c_init=1.0)),
    # 128^3 periodic box of the paper-mode analysis run (Sec. 4.2, 5.1): pore size of the
    # 256^3 workloads (shell 6 on 128 = shell 12 on 256), reaction directly r -> p at
    # one nucleation site per 64^3 block, xi = 1, sigma = 0.3, body force a = 3.616e-5
    # along x; tau is set from the Damkohler number by the analysis run
    "paper128": Workload("paper128", (128, 128, 128), 6, 0.5, 6, 0,
                         Params(tau=1.0, sigma=0.3, beta=0.7, theta_deg=90.0, accel=(3.616e-5, 0.0, 0.0),
                                reaction_mode=1, xi=1.0, k_rate=0.0)),
    # 96^3 column of the adjoint workload
    "column96": Workload("column96", (96, 96, 96), 6, 0.5, 5, 1,
                         Params(theta_deg=60.0, k_rate=2e-3, u_in=0.004, c_in=1.0)),
}


def batched_workload(n=64, seed0=100, draw_seed=4242):
    """64 independent columns of uneven size: cube edge uniform in 48..96, porosity
    uniform in [0.4, 0.6], contact angle uniform in [20, 120] degrees, inlet velocity
    uniform in [0.001, 0.01]; mask k uses GRF seed seed0 + k with shell |k| = edge/16.
    Returns (masks, params, bc_z, edges)."""
    u = synth.uniform01(draw_seed, 4 * n).reshape(n, 4)
    masks, params, edges = [], [], []
    for k in range(n):
        edge = 48 + int(u[k, 0] * 49)            # 48 .. 96
        edge = min(edge, 96)
        phi = 0.4 + 0.2 * u[k, 1]
        theta = 20.0 + 100.0 * u[k, 2]
        u_in = 0.001 + 0.009 * u[k, 3]
        masks.append(synth.grf_mask((edge, edge, edge), max(2, round(edge / 16)), phi, seed0 + k,
                                    periodic_z=False))
        params.append(Params(tau=1.0, sigma=0.01, beta=0.7, theta_deg=theta, k_rate=5e-3, diffusivity=0.05,
                             u_in=u_in, c_in=1.0, c_init=1.0))
        edges.append(edge)
    return masks, params, [1] * n, edges
