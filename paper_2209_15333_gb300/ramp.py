"""Compression-ramp runs (the paper's Table 8 flow, synthetic grids) and the
comparison of the plain FP64 hybrid method with the FP32-bulk / FP64-state
form driven by the learned sensor.

    python -m paper_2209_15333_gb300.ramp --case 4 [--steps 600] [--out result.json]

Case 4: Mach 2.9, 24 degrees, 1024 x 256 x 128, T_w/T_inf = 2.8,
T_ref = 108.1 K.  Case 5: Mach 6, 34 degrees, 1536 x 384 x 192, T_w = 5.9,
T_ref = 65 K.  Re_delta = 20000, Sutherland viscosity, hybrid scheme,
isothermal wall with a blowing/suction strip, inflow profile, extrapolation
at the outlet and the top, periodic span.  Wall pressure p_w/p_inf and skin
friction C_f = 2 tau_w (rho_inf = U_inf = 1) are averaged over the span and
over samples of the last quarter of the run.
"""
import argparse
import json
import sys
import time

import numpy as np

CASES = {
    4: dict(shape=(1024, 256, 128), angle=24.0, Ma=2.9, Tw=2.8, T_ref=108.1),
    5: dict(shape=(1536, 384, 192), angle=34.0, Ma=6.0, Tw=5.9, T_ref=65.0),
}
RE = 20000.0
BLOWING = dict(amp=0.02, x0=-15.0, x1=-10.0, omega=0.5, m=4, Lz=4.0)


def wall_quantities(U, met2, Ma, Tw, T_ref, gamma=1.4, Re=RE):
    """p_w/p_inf and C_f along the wall (span-averaged) from one state.

    C_f = 2 tau_w, tau_w = (mu_w/Re) du_t/dn with du_t/dn = |grad eta|
    d(u.t)/d eta at the wall (second-order one-sided; u_t = 0 at the wall),
    t the unit tangent along xi."""
    rho = U[0]
    u, v = U[1] / rho, U[2] / rho
    w = U[3] / rho
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * (u * u + v * v + w * w))
    pinf = 1.0 / (gamma * Ma * Ma)
    pw = p[:, 0, :].mean(axis=0) / pinf
    # tangent along the wall from the metrics: xi direction in x-y is
    # perpendicular to grad(eta); t = (eta_y, -eta_x)/|grad eta|
    ex, ey = met2[3, 0, :], met2[4, 0, :]
    ge = np.sqrt(ex * ex + ey * ey)
    tx, ty = ey / ge, -ex / ge
    ut = u * tx[None, None, :] + v * ty[None, None, :]
    dut = (4.0 * ut[:, 1, :] - ut[:, 2, :]) / 2.0 - 1.5 * ut[:, 0, :]
    s = 110.4 / T_ref
    mu_w = Tw ** 1.5 * (1.0 + s) / (Tw + s)
    cf = (2.0 * mu_w / Re * ge[None, :] * dut).mean(axis=0)
    return pw, cf


def van_driest(y, u, rho, mu_w, Re):
    """Van Driest transformed mean-velocity profile in wall units along one
    wall-normal line (y from the wall, y[0] = 0; u tangential velocity, rho
    density, span/time-averaged):
        u_VD = int_0^u sqrt(rho/rho_w) du,  u_tau = sqrt(tau_w/rho_w),
        tau_w = (mu_w/Re) du/dy|_w,  y+ = Re rho_w u_tau y / mu_w,
        u_VD+ = u_VD / u_tau
    (trapezoidal rule; du/dy at the wall second-order one-sided)."""
    y, u, rho = (np.asarray(a, dtype=np.float64) for a in (y, u, rho))
    h1, h2 = y[1] - y[0], y[2] - y[0]
    dudy = (u[1] * h2 * h2 - u[2] * h1 * h1 - u[0] * (h2 * h2 - h1 * h1)) / (h1 * h2 * (h2 - h1))
    tau_w = mu_w / Re * dudy
    rho_w = rho[0]
    u_tau = np.sqrt(abs(tau_w) / rho_w)
    w = np.sqrt(rho / rho_w)
    u_vd = np.concatenate([[0.0], np.cumsum(0.5 * (w[1:] + w[:-1]) * np.diff(u))])
    return Re * rho_w * u_tau * y / mu_w, u_vd / u_tau, u_tau


def station_profile(U, rc, x_station):
    """span-averaged density and tangential velocity along the eta line
    nearest to x_station, with the wall distance"""
    i = int(np.argmin(np.abs(rc["X"][0] - x_station)))
    rho = U[0, :, :, i].mean(axis=0)
    u = (U[1, :, :, i] / U[0, :, :, i]).mean(axis=0)
    y = rc["Y"][:, i] - rc["Y"][0, i]
    return y, u, rho


def case_shape(case, scale=1):
    nx, ny, nz = CASES[case]["shape"]
    return nx // scale, ny // scale, max(8, nz // scale)


def run(case, precision, learned, steps, sample_every, mlp_path=None, scale=1, scheme=3, **params):
    from . import build, cases
    from .solver import Solver
    from .train_sensor import load
    build.build()
    c = CASES[case]
    nx, ny, nz = case_shape(case, scale)
    rc = cases.ramp_case(nx, ny, nz, c["angle"], c["Ma"], Tw=c["Tw"])
    s = Solver((nx, ny, nz), rc["metrics2d"], bc_lo=(2, 1, 0), bc_hi=(3, 3, 0), precision=precision, scheme=scheme,
               Re=RE, Ma=c["Ma"], T_wall=c["Tw"], visc_law=0, T_ref=c["T_ref"], Pr=0.72, **params)
    s.set_inflow(rc["inflow"])
    s.set_blowing(BLOWING["amp"], BLOWING["x0"], BLOWING["x1"], BLOWING["omega"], BLOWING["m"], BLOWING["Lz"],
                  rc["wall_x"], rc["wall_z"])
    if learned:
        W, conf, _ = load(mlp_path) if mlp_path else load()
        s.set_sensor_mlp(W["w1"], W["w2"], W["w3"], W["b1"], W["b2"], W["b3"], conf_min=conf)
    s.set_state(rc["U"])
    return s, rc


def compare(case, steps, sample_every=None, mlp_path=None, scale=1, cfl=0.3):
    """Run the plain FP64 form and the mixed + learned form side by side."""
    import torch
    c = CASES[case]
    nx, ny, nz = case_shape(case, scale)
    N = nx * ny * nz
    sample_every = sample_every or max(1, steps // 40)
    out = {"case": case, "shape": [nx, ny, nz], "steps": steps, "Ma": c["Ma"], "angle": c["angle"],
           "resolution_scale": scale}
    ref, rc = run(case, 0, False, steps, sample_every, scale=scale)
    # dt is fixed from the initial field (reading R16); the CFL number must
    # leave room for the sound speed rise behind the shock that forms
    dt = ref.cfl_dt(cfl)
    out["dt"] = dt
    out["cfl_initial"] = cfl
    stats = {}
    for name, prec, learned in (("fp64_plain", 0, False), ("mixed_learned", 1, True), ("mixed_plain", 1, False)):
        s = ref if name == "fp64_plain" else run(case, prec, learned, steps, sample_every, mlp_path, scale)[0]
        pw_acc, cf_acc, nsamp = 0.0, 0.0, 0
        mis, unsafe, nmis, fallbacks = 0.0, 0.0, 0, 0
        t_gpu = 0.0
        start_avg = steps - steps // 4
        done = 0
        while done < steps:
            chunk = min(sample_every, steps - done)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step(dt, chunk)
            s.sync(3600.0)
            t_gpu += time.perf_counter() - t0
            done += chunk
            if done >= start_avg:
                U = s.get_state()
                pw, cf = wall_quantities(U, rc["metrics2d"], c["Ma"], c["Tw"], c["T_ref"])
                pw_acc = pw_acc + pw
                cf_acc = cf_acc + cf
                nsamp += 1
                if learned:
                    s.rhs(np.empty_like(U))
                    g = s.flags()
                    fallbacks += s.sensor_fallbacks()
                    s.set_sensor_mlp(None, None, None, None, None, None)
                    s.rhs(np.empty_like(U))
                    p = s.flags()
                    from .train_sensor import load
                    W, conf, _ = load(mlp_path) if mlp_path else load()
                    s.set_sensor_mlp(W["w1"], W["w2"], W["w3"], W["b1"], W["b2"], W["b3"], conf_min=conf)
                    mis += float((g != p).mean())
                    unsafe += float((g < p).mean())
                    nmis += 1
        rec = {"point_stage_per_s": N * 3 * steps / t_gpu, "pw": (pw_acc / nsamp).tolist(),
               "cf": (cf_acc / nsamp).tolist(), "samples": nsamp}
        if nmis:
            rec.update(misclassification=mis / nmis, unsafe_rate=unsafe / nmis,
                       fallback_fraction=fallbacks / (nmis * N))
        cls = s.flags()
        rec["class_fraction"] = (np.bincount(cls.ravel(), minlength=3)[:3] / cls.size).tolist()
        rec["gpu_seconds"] = t_gpu
        stats[name] = rec
        y, u, rho = station_profile(s.get_state(), rc, -5.0)
        sw = 110.4 / c["T_ref"]
        mu_w = c["Tw"] ** 1.5 * (1.0 + sw) / (c["Tw"] + sw)
        yp, up, utau = van_driest(y, u, rho, mu_w, RE)
        rec["van_driest_x-5"] = {"y_plus": yp.tolist(), "u_vd_plus": up.tolist(), "u_tau": float(utau)}
        if s is not ref:
            s.close()
    ref.close()
    base = stats["fp64_plain"]
    pw0, cf0 = np.array(base["pw"]), np.array(base["cf"])
    for name in ("mixed_learned", "mixed_plain"):
        pw1, cf1 = np.array(stats[name]["pw"]), np.array(stats[name]["cf"])
        stats[name]["pw_rel_l2_err"] = float(np.linalg.norm(pw1 - pw0) / np.linalg.norm(pw0))
        stats[name]["cf_rel_l2_err"] = float(np.linalg.norm(cf1 - cf0) / np.linalg.norm(cf0))
        stats[name]["pw_max_rel_err"] = float(np.abs(pw1 - pw0).max() / np.abs(pw0).max())
        stats[name]["cf_max_rel_err"] = float(np.abs(cf1 - cf0).max() / np.abs(cf0).max())
        stats[name]["speedup_vs_fp64"] = stats[name]["point_stage_per_s"] / base["point_stage_per_s"]
        u0 = np.array(base["van_driest_x-5"]["u_vd_plus"])
        u1 = np.array(stats[name]["van_driest_x-5"]["u_vd_plus"])
        stats[name]["u_vd_plus_max_rel_err"] = float(np.abs(u1 - u0).max() / np.abs(u0).max())
    out["results"] = stats
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", type=int, default=4, choices=[4, 5])
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--sample-every", type=int, default=0)
    ap.add_argument("--out", default="")
    ap.add_argument("--mlp", default="")
    ap.add_argument("--scale", type=int, default=1, help="divide the grid dimensions by this factor")
    ap.add_argument("--cfl", type=float, default=0.3, help="CFL number of the fixed dt on the initial field")
    a = ap.parse_args()
    res = compare(a.case, a.steps, a.sample_every or None, a.mlp or None, a.scale, a.cfl)
    summary = {k: v for k, v in res.items() if k != "results"}
    summary["results"] = {n: {k: v for k, v in r.items() if k not in ("pw", "cf", "van_driest_x-5")}
                          for n, r in res["results"].items()}
    print(json.dumps(summary))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f)


if __name__ == "__main__":
    sys.exit(main())
