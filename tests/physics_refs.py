"""Independent reference solutions used to pin the oracle: the exact
Riemann solver of the Euler equations (Toro 2009, Ch. 4) and the Sedov-Taylor
constant from the self-similar ODEs (Sedov 1959; Landau & Lifshitz Sec. 106).
Neither shares anything with the oracle or the CUDA path."""
import numpy as np


def exact_riemann(left, right, g, xi):
    """Exact solution of the 1-D Riemann problem at similarity coordinates
    xi = (x - x0)/t.  left/right = (rho, u, p).  Returns (rho, u, p) arrays
    and the star values (p*, u*, rho*_L, rho*_R)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)

    def f(p, r, pk, ck):
        if p > pk:  # shock
            A = 2.0 / ((g + 1) * r)
            B = (g - 1) / (g + 1) * pk
            return (p - pk) * np.sqrt(A / (p + B))
        return 2 * ck / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)

    from scipy.optimize import brentq
    ps = brentq(lambda p: f(p, rl, pl, cl) + f(p, rr, pr, cr) + ur - ul, 1e-12, 100.0,
                xtol=1e-15, rtol=1e-15)
    us = 0.5 * (ul + ur) + 0.5 * (f(ps, rr, pr, cr) - f(ps, rl, pl, cl))

    def rstar(r, pk):
        if ps > pk:
            q = ps / pk
            return r * (q + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * q + 1)
        return r * (ps / pk) ** (1 / g)

    rsl, rsr = rstar(rl, pl), rstar(rr, pr)
    xi = np.asarray(xi, float)
    rho, u, p = np.empty_like(xi), np.empty_like(xi), np.empty_like(xi)
    for t, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:
                sh = ul - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                rho[t], u[t], p[t] = (rl, ul, pl) if s < sh else (rsl, us, ps)
            else:
                head = ul - cl
                tail = us - cl * (ps / pl) ** ((g - 1) / (2 * g))
                if s < head:
                    rho[t], u[t], p[t] = rl, ul, pl
                elif s > tail:
                    rho[t], u[t], p[t] = rsl, us, ps
                else:
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    u[t] = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    rho[t] = rl * (c / cl) ** (2 / (g - 1))
                    p[t] = pl * (c / cl) ** (2 * g / (g - 1))
        else:
            if ps > pr:
                sh = ur + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                rho[t], u[t], p[t] = (rr, ur, pr) if s > sh else (rsr, us, ps)
            else:
                head = ur + cr
                tail = us + cr * (ps / pr) ** ((g - 1) / (2 * g))
                if s > head:
                    rho[t], u[t], p[t] = rr, ur, pr
                elif s < tail:
                    rho[t], u[t], p[t] = rsr, us, ps
                else:
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    u[t] = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    rho[t] = rr * (c / cr) ** (2 / (g - 1))
                    p[t] = pr * (c / cr) ** (2 * g / (g - 1))
    return (rho, u, p), (ps, us, rsl, rsr)


def sedov_xi0(g, j=2):
    """xi0 of R = xi0 (E t^2/rho0)^(1/5) for a point blast (j = 2: spherical),
    from the similarity ODEs in V, G, Z (v = (2r/5t)V, rho = rho0 G,
    c^2 = (2r/5t)^2 Z) integrated inward from the strong-shock jump
    conditions, and the energy integral
    1 = xi0^5 (16 pi/25) int_0^1 G (V^2/2 + Z/(g(g-1))) eta^4 d eta."""
    from scipy.integrate import solve_ivp
    alpha = 0.4

    def rhs(s, y):
        V, G, Z, _ = y
        A = np.array([[1.0, V - 1.0, 0.0],
                      [V - 1.0, Z / g, Z / g],
                      [0.0, (V - 1.0) * (1.0 - g), V - 1.0]])
        b = np.array([-(j + 1) * V, -V * V + V / alpha - 2 * Z / g, 2 / alpha - 2 * V])
        dV, dlnG, dlnZ = np.linalg.solve(A, b)
        eta = np.exp(s)
        return [dV, dlnG * G, dlnZ * Z, G * (0.5 * V * V + Z / (g * (g - 1))) * eta ** 5]

    y0 = [2 / (g + 1), (g + 1) / (g - 1), 2 * g * (g - 1) / (g + 1) ** 2, 0.0]
    sol = solve_ivp(rhs, [0.0, np.log(1e-4)], y0, rtol=1e-10, atol=1e-12, method="LSODA")
    integral = -sol.y[3, -1]
    return (25.0 / (16 * np.pi * integral)) ** 0.2
