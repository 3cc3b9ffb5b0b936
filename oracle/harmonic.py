"""Closed-form canonical energy of N non-interacting bosons in an isotropic 3-D
harmonic trap at finite bead number P (test infrastructure only).

The paper validates its simulations against "the analytical result" for trapped
bosons (appendix "Numerical Validation") without printing it.  This module
writes that result out for the primitive P-bead discretisation the sampler
uses, so the comparison carries no Trotter error:

* A cycle of k bosons is one ring of kP beads with spring constant m w_P^2
  (w_P = sqrt(P)/(beta hbar), Eq. eperm) and on-site potential
  (1/P)(1/2) m w0^2 r^2 per bead (the scaled potential U-bar of Eq.
  int-of-sum-all-permutations).  Diagonalising the cyclic chain gives, per
  Cartesian direction, z_k = 1 / (2 sinh(kP * asinh(beta hbar w0 / (2P)))).
* The cycle-type sum over permutations obeys the same recursion as Theorem
  forward-potential-recurrence integrated over positions:
  Z_0 = 1,  Z_n = (1/n) sum_{k=1}^{n} z_k Z_{n-k}  with z_k taken to the power 3.
* <E> = -d ln Z_N / d beta, evaluated analytically.

Units: m = hbar = 1 (the mass drops out of the partition-function ratio).
"""
import math


def _theta(beta, omega0, P):
    x = beta * omega0 / (2.0 * P)
    return math.asinh(x), (omega0 / (2.0 * P)) / math.sqrt(1.0 + x * x)


def _dlnZ(N, P, beta, omega0, dim, dth):
    """d ln Z_N / d lambda for a parameter lambda that enters only through
    theta, given dth = d theta / d lambda.

    Works with the rescaled y_k = z_k exp(dim k P theta) = (1 - exp(-2kP theta))^(-dim)
    and Y_n = Z_n exp(dim n P theta), which obey the same recursion and stay O(1).
    """
    th, _ = _theta(beta, omega0, P)
    y = [0.0] * (N + 1)
    dy = [0.0] * (N + 1)
    for k in range(1, N + 1):
        q = math.exp(-2.0 * k * P * th)
        y[k] = (1.0 - q) ** (-dim)
        # d/dlambda (1 - q)^(-dim) = -dim (1 - q)^(-dim-1) * (2 k P dth q)
        dy[k] = -dim * (1.0 - q) ** (-dim - 1) * (2.0 * k * P * dth * q)
    Y = [1.0] + [0.0] * N
    dY = [0.0] * (N + 1)
    for n in range(1, N + 1):
        s = ds = 0.0
        for k in range(1, n + 1):
            s += y[k] * Y[n - k]
            ds += dy[k] * Y[n - k] + y[k] * dY[n - k]
        Y[n] = s / n
        dY[n] = ds / n
    # ln Z_N = ln Y_N - dim N P theta
    return dY[N] / Y[N] - dim * N * P * dth


def mean_energy(N, P, beta, omega0=1.0, dim=3):
    """-d ln Z_N / d beta for N bosons, P beads, `dim` dimensions."""
    _, dth = _theta(beta, omega0, P)  # d theta / d beta
    return -_dlnZ(N, P, beta, omega0, dim, dth)


def mean_trap_energy(N, P, beta, omega0=1.0, dim=3):
    """<U-bar>, the mean trap energy (1/P) sum_j (1/2) m w0^2 |r_j|^2 of the same
    ensemble: U-bar is w0^2 times a positive function of the positions, so
    d ln Z / d w0 = -(2 beta / w0) <U-bar>, i.e. <U-bar> = -(w0 / (2 beta)) d ln Z / d w0."""
    x = beta * omega0 / (2.0 * P)
    dth = (beta / (2.0 * P)) / math.sqrt(1.0 + x * x)  # d theta / d w0
    return -(omega0 / (2.0 * beta)) * _dlnZ(N, P, beta, omega0, dim, dth)


def single_ring_partition(k, P, beta, omega0=1.0, dim=3):
    """z_k^dim: one ring of kP beads (k exchanged bosons)."""
    th, _ = _theta(beta, omega0, P)
    return (2.0 * math.sinh(k * P * th)) ** (-dim)


def partition_function(N, P, beta, omega0=1.0, dim=3):
    """Z_N by the cycle recursion (unscaled; small N only)."""
    Z = [1.0] + [0.0] * N
    for n in range(1, N + 1):
        Z[n] = sum(single_ring_partition(k, P, beta, omega0, dim) * Z[n - k]
                   for k in range(1, n + 1)) / n
    return Z[N]
