"""Random MPO Omega of Lemma 5.1 for the oracle (test infrastructure only).

Lemma 5.1 builds a J x K random matrix as a unit-rank MPO: Omega^(1) in R^{1 x J_1 x K x 1}
random, Omega^(i) in R^{1 x J_i x 1 x 1} random vectors for i >= 2, and Section 5.1 says the
entries are Gaussian. The paper fixes no generator, so both this oracle and the CUDA library
implement, each on its own, the same published counter-based stream:

  SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
    z_n = seed + (n + 1) * 0x9E3779B97F4A7C15  (mod 2^64)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;  z = (z ^ (z >> 27)) * 0x94D049BB133111EB;  z ^ (z >> 31)
  uniform u_n = ((z_n >> 11) + 1) * 2^-53, in (0, 1]
  normal g_m = sqrt(-2 ln u_{2m}) * cos(2 pi u_{2m+1})   (Box-Muller, cosine branch)

Draw order: Omega^(1) column-major (j fastest, then the K column index), then the vectors of
sites 2, 3, ..., d in turn. The libm used for log/cos may differ from CUDA's by an ulp, which
perturbs Omega at the 1e-16 level only.
"""

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, n0, count):
    """Outputs n0 .. n0+count-1 of the SplitMix64 stream started at ``seed`` (uint64 array)."""
    with np.errstate(over="ignore"):
        n = np.arange(n0 + 1, n0 + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + n * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniforms(seed, n0, count):
    z = splitmix64(seed, n0, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normals(seed, m0, count):
    """Gaussian draws m0 .. m0+count-1 (two uniforms per draw)."""
    u = uniforms(seed, 2 * m0, 2 * count)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def omega(seed, J, K):
    """Lemma 5.1 random MPO for column dims J = (J_1, ..., J_d) and K <= J_1 columns."""
    J = [int(j) for j in J]
    if K > J[0]:
        raise ValueError("Lemma 5.1 needs K <= J_1")
    g = normals(seed, 0, J[0] * K + sum(J[1:]))
    cores = [g[: J[0] * K].reshape(K, J[0]).T[None, :, :, None].copy()]  # (1, J1, K, 1)
    pos = J[0] * K
    for j in J[1:]:
        cores.append(g[pos:pos + j].reshape(1, j, 1, 1).copy())
        pos += j
    return cores
