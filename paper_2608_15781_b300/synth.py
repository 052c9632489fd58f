"""Seeded synthetic inputs: bicontinuous porous masks and initial fields.

This module holds input generators only -- none of the lattice Boltzmann
method's arithmetic -- so that the CUDA path and the CPU oracle can be fed the
very same inputs.

The paper's bijel-derived geometry (Sec. 3: a 256^3 subsample of a 1024^3
simulated bijel, porosity ~0.6, mean pore radius ~9 lattice units) is not
available, so a Gaussian random field band-passed to a spherical shell in
Fourier space and thresholded to the target porosity stands in for it: such
level sets of a narrow-band field are bicontinuous, like spinodal/bijel
structures.  Steps:

1. white Gaussian noise from SplitMix64 (Steele, Lea and Flood 2014) fed to the
   Box-Muller transform, one counter per lattice node;
2. FFT, keep the modes with |k| in [k0 - 1, k0 + 1], where |k| counts cycles
   per length of the shortest box edge (k_a = n_a * N_min / N_a), inverse FFT;
3. the porosity * N lowest values become fluid (ties broken by linear index);
4. artefact cleanup as in Sec. 3: keep the largest 6-connected fluid and the
   largest 6-connected solid component, flip every other component.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, n):
    """The first ``n`` outputs of SplitMix64 started at ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        x = np.uint64(seed) + _GOLDEN * np.arange(1, n + 1, dtype=np.uint64)
        x = (x ^ (x >> np.uint64(30))) * _M1
        x = (x ^ (x >> np.uint64(27))) * _M2
        x = x ^ (x >> np.uint64(31))
    return x


def uniform01(seed, n):
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian_noise(seed, shape):
    """Standard normal field by Box-Muller on consecutive SplitMix64 pairs."""
    n = int(np.prod(shape))
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
    return z[:n].reshape(shape)


def shell_filtered_field(shape, k0, seed):
    """Gaussian random field band-passed to |k| in [k0-1, k0+1] (shape = (nz, ny, nx))."""
    noise = gaussian_noise(seed, shape)
    nmin = min(shape)
    ks = [np.fft.fftfreq(n) * n * (nmin / n) for n in shape]
    kz, ky, kx = np.meshgrid(*ks, indexing="ij")
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    band = (kmag >= k0 - 1) & (kmag <= k0 + 1)
    return np.real(np.fft.ifftn(np.fft.fftn(noise) * band))


def _label_periodic(mask, periodic_z):
    """6-connected component labels of ``mask`` with periodic x, y (and z if asked)."""
    from scipy import ndimage

    lab, n = ndimage.label(mask)
    if n == 0:
        return lab, 0
    parent = np.arange(n + 1)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    def join(a_face, b_face):
        both = (a_face > 0) & (b_face > 0)
        for a, b in zip(a_face[both].ravel(), b_face[both].ravel()):
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)

    join(lab[:, :, 0], lab[:, :, -1])
    join(lab[:, 0, :], lab[:, -1, :])
    if periodic_z:
        join(lab[0], lab[-1])
    roots = np.array([find(a) for a in range(n + 1)])
    return roots[lab], n


def _keep_largest(mask, periodic_z):
    lab, n = _label_periodic(mask, periodic_z)
    if n <= 1:
        return mask
    counts = np.bincount(lab.ravel())
    counts[0] = 0
    keep = int(np.argmax(counts))
    return lab == keep


def grf_mask(shape, k0, porosity, seed, periodic_z=True, cleanup=True):
    """Bicontinuous solid mask (True = solid), shape = (nz, ny, nx), x fastest in memory."""
    field = shell_filtered_field(shape, k0, seed).ravel()
    n = field.size
    order = np.argsort(field, kind="stable")
    fluid = np.zeros(n, dtype=bool)
    fluid[order[: int(round(porosity * n))]] = True
    fluid = fluid.reshape(shape)
    if cleanup:
        fluid = _keep_largest(fluid, periodic_z)
        solid = _keep_largest(~fluid, periodic_z)
        fluid = ~solid
    return np.ascontiguousarray(~fluid)


def droplet_fields(shape, center, radius, width=2.0, inside_r=True):
    """Densities (rho_r, rho_p) of a diffuse sphere of radius ``radius`` (tanh profile)."""
    nz, ny, nx = shape
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    phi = np.tanh((radius - r) / width)
    if not inside_r:
        phi = -phi
    return (1.0 + phi) / 2.0, (1.0 - phi) / 2.0
