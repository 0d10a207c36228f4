"""Closed forms of the discrete scheme that the tests compare the oracle and
the GPU kernels with (test infrastructure; no part of the method's code path).
"""
import math

import numpy as np


def standing_wave_amplitudes(nx, ny, mx, my, H, dx, dt, theta, steps, g=9.81):
    """Amplitude of the cosine mode after 1 .. steps steps, per unit of the start's.

    With n = 0 and a small disturbance eps of a flat surface H, h_f = H + O(eps)
    and Eq. 3-4 reduce to the linear staggered scheme
        q' = gamma q - g H dt/dx (h_R - h_L),   h' = h - dt/dx (sum of the new faces out),
    gamma the theta weighting's factor on a sine mode of the faces,
    theta + (1 - theta) cos(k dx) (1 for Eq. 3 as printed).  On the mode
    h = A cos(kx x) cos(ky y), qx = Bx sin(kx x) cos(ky y), qy = By cos(kx x) sin(ky y)
    (the walls are nodes of the sines), with s_i = 2 sin(k_i dx / 2) dt / dx:
        Bx' = gamma_x Bx + g H s_x A,  By' = gamma_y By + g H s_y A,  A' = A - s_x Bx' - s_y By'.
    For theta = 1 the matrix has determinant 1 and trace 2 cos(phi) with
    sin(phi / 2) = sqrt(g H) dt/dx sqrt(sin^2(kx dx/2) + sin^2(ky dx/2)) (the
    scheme's dispersion relation), so A_n = sin(n phi)/sin(phi) (1 - g H s^2)
    - sin((n - 1) phi)/sin(phi); otherwise the recurrence is iterated."""
    kx, ky = math.pi * mx / (nx * dx), math.pi * my / (ny * dx)
    sx, sy = 2 * math.sin(kx * dx / 2) * dt / dx, 2 * math.sin(ky * dx / 2) * dt / dx
    c = g * H
    if theta == 1.0:
        s2 = sx * sx + sy * sy
        phi = math.acos(1.0 - 0.5 * c * s2)
        n = np.arange(1, steps + 1)
        return (np.sin(n * phi) * (1.0 - c * s2) - np.sin((n - 1) * phi)) / math.sin(phi)
    gx, gy = theta + (1 - theta) * math.cos(kx * dx), theta + (1 - theta) * math.cos(ky * dx)
    M = np.array([[1.0 - c * (sx * sx + sy * sy), -sx * gx, -sy * gy],
                  [c * sx, gx, 0.0],
                  [c * sy, 0.0, gy]])
    v, out = np.array([1.0, 0.0, 0.0]), []
    for _ in range(steps):
        v = M @ v
        out.append(v[0])
    return np.array(out)
