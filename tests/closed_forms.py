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


def standing_wave_modes(nx, ny, mx, my, dx):
    """The cosine mode of the depths and the sine modes of the x- and y-face
    discharges that go with it (walls at the nodes of the sines): arrays of the
    cells' (ny, nx), the x-faces' (ny, nx + 1) and the y-faces' (ny + 1, nx) shapes."""
    kx, ky = math.pi * mx / (nx * dx), math.pi * my / (ny * dx)
    xc, yc = (np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx
    xf, yf = np.arange(nx + 1) * dx, np.arange(ny + 1) * dx
    return (np.outer(np.cos(ky * yc), np.cos(kx * xc)), np.outer(np.cos(ky * yc), np.sin(kx * xf)),
            np.outer(np.sin(ky * yf), np.cos(kx * xc)))


def standing_wave_matrix(nx, ny, mx, my, H, dx, dt, theta, g=9.81):
    """One step of the linearised scheme on the mode amplitudes (A, Bx, By) of
    standing_wave_modes (the recurrence in standing_wave_amplitudes)."""
    kx, ky = math.pi * mx / (nx * dx), math.pi * my / (ny * dx)
    sx, sy = 2 * math.sin(kx * dx / 2) * dt / dx, 2 * math.sin(ky * dx / 2) * dt / dx
    gx, gy = theta + (1 - theta) * math.cos(kx * dx), theta + (1 - theta) * math.cos(ky * dx)
    c = g * H
    return np.array([[1.0 - c * (sx * sx + sy * sy), -sx * gx, -sy * gy],
                     [c * sx, gx, 0.0],
                     [c * sy, 0.0, gy]])


def standing_wave_gradient(nx, ny, mx, my, H, dx, dt, theta, steps):
    """dL/d(h0, qx0, qy0) of L = <mode, depths after `steps` steps> for a lake at
    rest (depth H, no discharge), where the scheme's Jacobian is the linear one.

    The transposed step keeps the mode subspace, so dL/dh0 = (M^n)_00 mode and,
    on interior faces, dL/dq0 = (M^n)_0b |mode|^2 / |s_b|^2 s_b for the sine
    modes s_b of the two axes.  A wall face's old value enters only the theta
    numerator of the interior face next to it in the first step (weight
    (1 - theta)/2), so its gradient is that weight times the adjoint of that
    face's new value in step 1: lambda_q + dt/dx (lambda_R - lambda_L) with the
    (n - 1)-step gradients lambda."""
    mh, mqx, mqy = standing_wave_modes(nx, ny, mx, my, dx)
    M = standing_wave_matrix(nx, ny, mx, my, H, dx, dt, theta)
    R, R1 = np.linalg.matrix_power(M, steps)[0], np.linalg.matrix_power(M, steps - 1)[0]
    nh, w, r = float(np.sum(mh * mh)), 0.5 * (1.0 - theta), dt / dx
    gh = R[0] * mh
    gx = np.zeros_like(mqx)
    gy = np.zeros_like(mqy)
    if nx > 1:
        gx = R[1] * nh / float(np.sum(mqx * mqx)) * mqx
        a1 = R1[1] * nh / float(np.sum(mqx * mqx))
        gx[:, 0] = w * (a1 * mqx[:, 1] + r * R1[0] * (mh[:, 1] - mh[:, 0]))
        gx[:, nx] = w * (a1 * mqx[:, nx - 1] + r * R1[0] * (mh[:, nx - 1] - mh[:, nx - 2]))
    if ny > 1:
        gy = R[2] * nh / float(np.sum(mqy * mqy)) * mqy
        a1 = R1[2] * nh / float(np.sum(mqy * mqy))
        gy[0, :] = w * (a1 * mqy[1, :] + r * R1[0] * (mh[1, :] - mh[0, :]))
        gy[ny, :] = w * (a1 * mqy[ny - 1, :] + r * R1[0] * (mh[ny - 1, :] - mh[ny - 2, :]))
    return mh, gh, gx, gy
