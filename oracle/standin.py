"""Seeded state-transition stand-in for the physics simulator (NOT the paper's method).

Test infrastructure only.  The paper runs PhysX inside Isaac Gym (Sec. 2, App. A.1); the
simulator is outside the method, so a seeded linear stochastic transition takes its place.
It is *defined* as an fp32 recurrence with a fixed operation order and no fused
multiply-add, so that the CUDA path (which uses explicit round-to-nearest fp32 intrinsics)
produces the same bits.  Every constant is a dyadic rational (exact in fp32) except the
ones that come from the config (sim_dt, gains), which both sides round from the same
double to fp32.  Innovations xi are Irwin-Hall(4) normals (oracle.rng), exact on both
sides.  parity unpinned: no passage of the paper defines this transition.

Per substep k (slots 32k + j of the env's key), with tau the PD torque of Sec. 3.2:
    qd <- (A_Q qd + sim_dt (INV_I tau)) + S_Q xi           q <- q + sim_dt qd
    v_x <- (RHO_V v_x + (1 - RHO_V) v*_x) + S_V xi          (v_y likewise, v_z without target)
    w_x <- RHO_W w_x + S_W xi, w_y likewise; w_z <- (RHO_W w_z + (1 - RHO_W) w*_z) + S_W xi
    heading (c, s) rotated by w_z sim_dt to first order and renormalised
    p <- p + sim_dt R(c, s) v_xy                            (p is relative to the spawn origin)
    g_x, g_y <- RHO_G g + S_G xi;   g_z = -sqrt(max(0, 1 - g_x^2 - g_y^2))
    z <- (RHO_Z z + (1 - RHO_Z) z_nom(level)) + S_Z xi,     z_nom = 0.5 + 0.0625 level
"""
import numpy as np

from . import rng

f32 = np.float32

A_Q = f32(0.96875)
INV_I = f32(2.0)
S_Q = f32(0.0625)
RHO_V = f32(0.96875)
ONE_M_RHO_V = f32(0.03125)
S_V = f32(0.03125)
RHO_W = f32(0.96875)
ONE_M_RHO_W = f32(0.03125)
S_W = f32(0.0625)
RHO_G = f32(0.96875)
S_G = f32(0.0078125)
RHO_Z = f32(0.96875)
ONE_M_RHO_Z = f32(0.03125)
S_Z = f32(0.00390625)
Z_NOM0 = f32(0.5)
Z_NOM_PER_LEVEL = f32(0.0625)


def z_nominal(level):
    return (level.astype(f32) * Z_NOM_PER_LEVEL + Z_NOM0).astype(f32)


def substep(S, tau, k, key, sim_dt):
    """Advance the fp32 state dict S in place by one substep; tau is [12, N] fp32."""
    dts = f32(sim_dt)
    base = 32 * k

    def xi(j):
        return rng.irwin_hall_f32(rng.word(key, base + j))

    for j in range(12):
        qd = (A_Q * S["qd"][j] + dts * (INV_I * tau[j])) + S_Q * xi(j)
        S["qd"][j] = qd
        S["q"][j] = S["q"][j] + dts * qd
    S["vx"] = (RHO_V * S["vx"] + ONE_M_RHO_V * S["cmdx"]) + S_V * xi(12)
    S["vy"] = (RHO_V * S["vy"] + ONE_M_RHO_V * S["cmdy"]) + S_V * xi(13)
    S["vz"] = RHO_V * S["vz"] + S_V * xi(14)
    S["wx"] = RHO_W * S["wx"] + S_W * xi(15)
    S["wy"] = RHO_W * S["wy"] + S_W * xi(16)
    S["wz"] = (RHO_W * S["wz"] + ONE_M_RHO_W * S["cmdw"]) + S_W * xi(17)
    w = S["wz"] * dts
    c1 = S["hc"] - S["hs"] * w
    s1 = S["hs"] + S["hc"] * w
    n = np.sqrt(c1 * c1 + s1 * s1)
    S["hc"] = c1 / n
    S["hs"] = s1 / n
    dx = S["hc"] * S["vx"] - S["hs"] * S["vy"]
    dy = S["hs"] * S["vx"] + S["hc"] * S["vy"]
    S["px"] = S["px"] + dts * dx
    S["py"] = S["py"] + dts * dy
    S["gx"] = RHO_G * S["gx"] + S_G * xi(18)
    S["gy"] = RHO_G * S["gy"] + S_G * xi(19)
    S["gz"] = -np.sqrt(np.maximum(f32(0.0), f32(1.0) - (S["gx"] * S["gx"] + S["gy"] * S["gy"])))
    S["z"] = (RHO_Z * S["z"] + ONE_M_RHO_Z * z_nominal(S["level"])) + S_Z * xi(20)
    for name in ("vx", "vy", "vz", "wx", "wy", "wz", "hc", "hs", "px", "py", "gx", "gy", "gz", "z"):
        assert S[name].dtype == np.float32, name
