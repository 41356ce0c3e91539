"""FP64 oracle of the Newmark-beta time stepping of the structure (test
infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and never by the product path.

The structure's semi-discretisation in time (Sec. 4.1.2) uses the Newmark-beta
method.  Its definition, for displacement d, velocity v and acceleration a:

    d_n = d_(n-1) + dt v_(n-1) + dt^2/2 ((1 - 2 beta) a_(n-1) + 2 beta a_n)
    v_n = v_(n-1) + dt ((1 - gamma) a_(n-1) + gamma a_n)

Solved for the new acceleration, the first line gives a_n from d_n, so the
inertia force rho a_n of step n splits into rho / (beta dt^2) d_n (the part
that enters the tangent) minus rho h_(n-1), with the history

    h = d / (beta dt^2) + v / (beta dt) + (1 - 2 beta) / (2 beta) a

of the previous step.  ``newmark_update`` is that bookkeeping; ``sdof`` runs
the method on the single-degree-of-freedom oscillator m u'' + k u = 0 (the
implicit step (k + m c) u_n = m h_(n-1), c = 1 / (beta dt^2)), which the pins
compare with closed forms.
"""
from __future__ import annotations

import numpy as np


def newmark_update(d_new, d_old, v_old, a_old, beta, gamma, dt):
    """a_n, v_n and the history h_n after the solve of step n (Sec. 4.1.2)."""
    a_new = (d_new - d_old) / (beta * dt * dt) - v_old / (beta * dt) - (1.0 - 2.0 * beta) / (2.0 * beta) * a_old
    v_new = v_old + dt * ((1.0 - gamma) * a_old + gamma * a_new)
    hist = d_new / (beta * dt * dt) + v_new / (beta * dt) + (1.0 - 2.0 * beta) / (2.0 * beta) * a_new
    return a_new, v_new, hist


def sdof(m, k, u0, v0, dt, n_steps, beta, gamma):
    """Displacements, velocities and energies 1/2 m v^2 + 1/2 k u^2 of the
    free oscillator integrated by Newmark-beta from (u0, v0)."""
    c = 1.0 / (beta * dt * dt)
    u, v = float(u0), float(v0)
    a = -k * u / m
    hist = u * c + v / (beta * dt) + (1.0 - 2.0 * beta) / (2.0 * beta) * a
    us, vs, es = [u], [v], [0.5 * m * v * v + 0.5 * k * u * u]
    for _ in range(n_steps):
        u_new = m * hist / (k + m * c)
        a, v, hist = newmark_update(u_new, u, v, a, beta, gamma, dt)
        u = u_new
        us.append(u)
        vs.append(v)
        es.append(0.5 * m * v * v + 0.5 * k * u * u)
    return np.array(us), np.array(vs), np.array(es)
