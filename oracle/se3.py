"""SE(3) pose increments of the differentiable rendering, in FP64 -- TEST INFRASTRUCTURE ONLY.

The optimisation of §III-C refines keyframe poses together with the map; the renderer's pose
gradient is taken with respect to a left increment xi = (rho, phi) of the world-to-camera
pose, T_cw <- Exp(xi) T_cw (rho: translation part, phi: rotation part).

  hat(xi)            the 4 x 4 matrix [[phi^, rho], [0, 0]] of se(3)
  exp(xi)            Exp(xi) = the matrix exponential of hat(xi) (scipy.linalg.expm)
  left_jacobian(xi)  the 6 x 6 J with Exp(xi + d) = Exp(J d) Exp(xi) to first order, from its
                     definition J[:, k] = vee(dExp(xi)[e_k] Exp(xi)^-1), the directional
                     derivative dExp of the matrix exponential being the exact Frechet
                     derivative read off the exponential of the block matrix
                     [[hat(xi), hat(e_k)], [0, hat(xi)]]
  twist_grad(xi, g)  J(xi)^T g: the gradient with respect to xi of a function whose gradient
                     with respect to a left increment at Exp(xi) T is g
  move_camera(c, xi) the camera dict with (R, t) replaced by Exp(xi) (R, t)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def hat(xi):
    rho, phi = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    M[:3, 3] = rho
    return M


def vee(M):
    return np.array([M[0, 3], M[1, 3], M[2, 3], M[2, 1], M[0, 2], M[1, 0]])


def exp(xi):
    return scipy.linalg.expm(hat(xi))


def left_jacobian(xi):
    A = hat(xi)
    Einv = np.linalg.inv(scipy.linalg.expm(A))
    J = np.zeros((6, 6))
    for k in range(6):
        e = np.zeros(6)
        e[k] = 1.0
        B = np.zeros((8, 8))
        B[:4, :4] = A
        B[4:, 4:] = A
        B[:4, 4:] = hat(e)
        D = scipy.linalg.expm(B)[:4, 4:]        # Frechet derivative of expm at A along hat(e_k)
        J[:, k] = vee(D @ Einv)
    return J


def twist_grad(xi, g_left):
    return left_jacobian(xi).T @ np.asarray(g_left, float)


def move_camera(cam, xi):
    T = np.eye(4)
    T[:3, :3] = np.asarray(cam["R"], float)
    T[:3, 3] = np.asarray(cam["t"], float)
    T2 = exp(xi) @ T
    c = dict(cam)
    c["R"], c["t"] = T2[:3, :3].copy(), T2[:3, 3].copy()
    return c
