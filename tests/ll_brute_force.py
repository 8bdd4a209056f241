"""Brute-force RK4 integration of the Landau-Lifshitz equation of motion of an
electron in a linearly polarised plane-wave pulse (test helper, no oracle code).

Normalised units: time in 1/omega0, length in c/omega0, momentum in m c,
fields in m c omega0 / e.  The laser moves along +z with phase phi = t - z,
vector potential A_x = psi(phi) = a0 G(phi) sin(phi), so E = (-psi', 0, 0) and
B = (0, -psi', 0).  The LL force (Landau & Lifshitz, Classical Theory of
Fields, Sec. 76) for a charge -e, with tau = (2/3) R_c, R_c = r_e omega0 / c:

  du/dt = -(E + v x B)
          + tau * ( -gamma (1 - v_z) (E' + v x B')
                    + E x B + B x (B x v) + E (v . E)
                    - gamma^2 v [ (E + v x B)^2 - (E . v)^2 ] )

where ' is d/dphi (the convective derivative of a plane-wave field along the
trajectory is (1 - v_z) d/dphi).
"""
import numpy as np


def psi_derivs(phi, a0, Phi):
    """psi' and psi'' for psi = a0 G sin(phi), G = exp(-2 ln2 (phi/Phi)^2)."""
    c = 2.0 * np.log(2.0) / Phi ** 2
    G = np.exp(-c * phi * phi)
    G1 = -2.0 * c * phi * G
    G2 = (4.0 * c * c * phi * phi - 2.0 * c) * G
    s, co = np.sin(phi), np.cos(phi)
    p1 = a0 * (G1 * s + G * co)
    p2 = a0 * (G2 * s + 2.0 * G1 * co - G * s)
    return p1, p2


def integrate(gamma0, a0, Phi, Rc, steps_per_cycle=200, span=3.0):
    """Integrate from phi = -span*Phi to +span*Phi.  Vectorised over cases.

    Returns (h0, h_final, gamma_final, ux_final, uz_final) with
    h = gamma - u_z, the light-front momentum.
    """
    gamma0 = np.atleast_1d(np.asarray(gamma0, dtype=np.float64))
    a0 = np.broadcast_to(np.asarray(a0, dtype=np.float64), gamma0.shape).copy()
    tau = (2.0 / 3.0) * Rc
    uz0 = -np.sqrt(gamma0 ** 2 - 1.0)
    # y = (t, z, ux, uy, uz); x, y positions do not enter plane-wave fields
    t = np.zeros_like(gamma0)
    z = np.full_like(gamma0, span * Phi)       # phi = t - z = -span*Phi
    ux = np.zeros_like(gamma0)
    uy = np.zeros_like(gamma0)
    uz = uz0.copy()

    def f(t, z, ux, uy, uz):
        g = np.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
        vx, vy, vz = ux / g, uy / g, uz / g
        p1, p2 = psi_derivs(t - z, a0, Phi)
        Ex, By = -p1, -p1
        dEx, dBy = -p2, -p2
        # v x B with B = (0, By, 0): (vy*0 - vz*By, vz*0 - vx*0, vx*By - vy*0)
        vxB = (-vz * By, 0.0 * vx, vx * By)
        vxdB = (-vz * dBy, 0.0 * vx, vx * dBy)
        F = (Ex + vxB[0], vxB[1], vxB[2])          # E + v x B
        lor = (-F[0], -F[1], -F[2])
        # E x B = (0*0 - 0*By, 0*0 - Ex*0, Ex*By - 0*0)
        ExB = (0.0 * vx, 0.0 * vx, Ex * By)
        # B x (B x v): B x v = (By*vz - 0, 0*vx - 0*vz, 0*vy - By*vx)
        Bxv = (By * vz, 0.0 * vx, -By * vx)
        BxBxv = (By * Bxv[2] - 0.0, 0.0 * Bxv[0] - 0.0 * Bxv[2], 0.0 - By * Bxv[0])
        vE = vx * Ex
        E_vE = (Ex * vE, 0.0 * vx, 0.0 * vx)
        F2 = F[0] ** 2 + F[1] ** 2 + F[2] ** 2 - vE * vE
        k1 = (1.0 - vz)
        rr = [-g * k1 * (dEx * (c == 0) + vxdB[c]) + ExB[c] + BxBxv[c] + E_vE[c] - g * g * (vx, vy, vz)[c] * F2
              for c in range(3)]
        return (np.ones_like(t), vz,
                lor[0] + tau * rr[0], lor[1] + tau * rr[1], lor[2] + tau * rr[2])

    # phase advances ~2 per unit time; steps_per_cycle per 2 pi of phase
    dt = np.pi / steps_per_cycle
    phi_end = span * Phi
    nsteps = int(np.ceil((2.0 * span * Phi) / 2.0 / dt)) + 10
    for _ in range(nsteps):
        k1 = f(t, z, ux, uy, uz)
        y1 = [v + 0.5 * dt * k for v, k in zip((t, z, ux, uy, uz), k1)]
        k2 = f(*y1)
        y2 = [v + 0.5 * dt * k for v, k in zip((t, z, ux, uy, uz), k2)]
        k3 = f(*y2)
        y3 = [v + dt * k for v, k in zip((t, z, ux, uy, uz), k3)]
        k4 = f(*y3)
        t, z, ux, uy, uz = [v + dt / 6.0 * (a + 2 * b + 2 * c + d)
                            for v, a, b, c, d in zip((t, z, ux, uy, uz), k1, k2, k3, k4)]
        if np.all(t - z > phi_end):
            break
    g = np.sqrt(1.0 + ux * ux + uy * uy + uz * uz)
    h0 = gamma0 - uz0
    hf = g - uz
    return h0, hf, g, ux, uz
