"""Seeded synthetic workloads of the boundary-layer dispersion problem.

This module holds scenario parameters, level schedules and seeds only -- no
arithmetic of the method -- so both the CUDA path and the CPU oracle can be
driven from the same inputs.  It imports nothing from the rest of the package.

Scenarios
---------
``BL600``   the neutral boundary layer with u* = 0.2 m/s, f = 1e-4 1/s,
            H = 0.3 u*/f = 600 m, sigma_w = 1.3 u* (1 - z/H)^(3/4),
            tau = 0.5 z / sigma_w / (1 + 15 f z / u*), eps_reg = 1e-3 H,
            release at z0 = 0.1 H with w0 ~ N(0, sigma_w(z0)^2), T = 600 s,
            QoIs z(T) and 1[z(T) < 0.1 H].
``PAPER``   the nondimensional scenario of the paper's experiments (Section
            5): H = 1 (1 km), u* = 0.2, T = 1 (1000 s), X0 = 0.05, U0 = 0.1,
            eps_reg = 0.01, tau = 0.5 X / sigma_U (no Coriolis factor).
"""

SE, GL, BAOAB = 0, 1, 2
INTEGRATORS = {"se": SE, "gl": GL, "baoab": BAOAB}

BL600 = dict(
    u_star=0.2, f_coriolis=1e-4, H=600.0, kappa_sigma=1.3, kappa_tau=0.5, c_f=15.0,
    eps_reg_frac=1e-3, z0=60.0, w0=0.0, w0_mode=1, T=600.0, M0=8, level_min=0, L_max=10,
    qoi_threshold=60.0, coupling=0, drift_outside=0, n_init=10000, stream_id=0,
)

PAPER = dict(
    u_star=0.2, f_coriolis=1e-4, H=1.0, kappa_sigma=1.3, kappa_tau=0.5, c_f=0.0,
    eps_reg_frac=0.01, z0=0.05, w0=0.1, w0_mode=0, T=1.0, M0=40, level_min=0, L_max=10,
    qoi_threshold=0.1555, coupling=0, drift_outside=0, n_init=10000, stream_id=0,
)

# Symplectic Euler needs h < 2 / lambda_max; with eps_reg = 0.6 m in BL600 that
# is M >= 261 steps over 600 s, i.e. level 6 (512 steps) and finer.
SE_LEVEL_MIN_BL600 = 6


def bl600(integrator=GL, **overrides):
    """BL600 parameters for one integrator (SE starts at its stable level)."""
    d = dict(BL600)
    if integrator == SE:
        d["level_min"] = SE_LEVEL_MIN_BL600
    d.update(overrides)
    return d


def well_mixed(**overrides):
    """BL600 started from the well-mixed state z ~ U(0, H), w ~ N(0, sigma_w(z)^2)."""
    d = dict(BL600, w0_mode=2)
    d.update(overrides)
    return d


def schedule_c4(levels=13, n0=1e9, decay=10 ** -0.5, level_min=0):
    """Batched multi-level workload: N_l = n0 * decay^l paths on levels
    level_min..levels-1 (1e9 on level 0 down to 1e3 on level 12)."""
    out = []
    for l in range(level_min, levels):
        out.append((l, int(round(n0 * decay ** l))))
    return out


SEED = 1
