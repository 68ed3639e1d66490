"""Named, seeded workloads (the synthetic stand-ins for the paper's floor-plan experiments).

Each workload is a plain dict of sizes and noise settings plus a seed; `make_map` and
`make_walk` turn it into inputs.  Nothing here computes any part of the filter.

* ``rooms64``      64 x 64 cells of 0.1 m, K = 16 bins, 4 x 4 rooms; 200 steps at dt 0.1 s.
* ``office512``    512 x 512 cells of 0.05 m, K = 64 bins; office plan; 2000 steps at dt 0.01 s.
* ``office512_aniso`` the same map, bins and walk with anisotropic motion noise (Eq. 6): sigma
                   1.0 cell along each bin's heading, 0.5 across it.
* ``office512_dense`` the office512 session with a dense scan update (Eq. 9 on every state):
                   a 384-direction expected-range table (6 per bin, r_max 10 m) and a 360-beam
                   scan (every 4th beam scored, sigma 0.1 m) after every step.
* ``office2048``   2048 x 2048 cells of 0.05 m, K = 72 bins, BF16 storage; a 360-beam scan every
                   10th step; parity on a 256 x 256 crop.
* ``batch64``      64 sessions, side log-uniform in [128, 1024], K in {36, 48, 64, 72}.
* ``serve256``     256 sessions on 10 maps, side log-uniform in [256, 2048], K in [36, 72] (x4).

Common settings: motion-noise sigma 0.5 cell in x/y and 1 bin in theta; odometry noise 2 % of
the translation per component and 0.01 rad in heading; speed U(0.3, 0.6) m/s, yaw rate
U(-0.5, 0.5) rad/s redrawn every second.
"""
from __future__ import annotations

import math

import numpy as np

from . import floorplan, trajectory

COMMON = dict(sigma_xy_cells=0.5, sigma_theta_bins=1.0, trans_noise_frac=0.02,
              rot_sigma=0.01)

WORKLOADS = {
    "rooms64": dict(COMMON, name="rooms64", seed=0, H=64, W=64, K=16, cell=0.1,
                    steps=200, dt=0.1, storage="f32", plan="rooms"),
    "office512": dict(COMMON, name="office512", seed=1, H=512, W=512, K=64, cell=0.05,
                      steps=2000, dt=0.01, storage="f32", plan="office"),
    "office512_aniso": dict(COMMON, name="office512_aniso", seed=1, H=512, W=512, K=64, cell=0.05,
                            steps=2000, dt=0.01, storage="f32", plan="office", sigma_xy_cells=1.0,
                            sigma_cross_cells=0.5),
    "office512_dense": dict(COMMON, name="office512_dense", seed=1, H=512, W=512, K=64, cell=0.05,
                            steps=2000, dt=0.01, storage="f32", plan="office", n_angles=384,
                            r_max=10.0, n_beams=360, angle_min=-math.pi, angle_inc=math.pi / 180,
                            beam_stride=4, sigma_r=0.1, scan_noise=0.05, dropout=0.05),
    "office2048": dict(COMMON, name="office2048", seed=2, H=2048, W=2048, K=72, cell=0.05,
                       steps=1000, dt=0.01, storage="bf16", plan="office", scan_every=10,
                       n_beams=360, angle_inc=math.pi / 180, r_max=10.0, scan_noise=0.05,
                       dropout=0.05, beam_stride=4, sigma_r=0.1, n_samples=4096, crop=256),
    "batch64": dict(COMMON, name="batch64", seed=3, n_sessions=64, side=(128, 1024),
                    ks=(36, 48, 64, 72), cell=0.05, steps=2000, dt=0.01, storage="bf16",
                    plan="office"),
    "serve256": dict(COMMON, name="serve256", seed=4, n_sessions=256, n_maps=10, side=(256, 2048),
                     ks=tuple(range(36, 73, 4)), cell=0.05, dt=0.01, odom_hz=100.0, scan_hz=10.0,
                     storage="bf16", plan="office", hbm_budget_gb=120.0, min_shift_cells=1.0,
                     n_beams=360, angle_inc=math.pi / 180, r_max=10.0, scan_noise=0.05,
                     dropout=0.05, beam_stride=4, sigma_r=0.1, n_samples=1024),
}


def get(name: str) -> dict:
    return dict(WORKLOADS[name])


def make_map(wl: dict) -> np.ndarray:
    if wl["plan"] == "rooms":
        return floorplan.rooms_map(wl["seed"], size=wl["H"])
    return floorplan.office_map(wl["seed"], size=wl["H"], cell=wl["cell"])


def make_walk(wl: dict, occ: np.ndarray, steps: int | None = None, seed_offset: int = 0):
    return trajectory.random_walk(occ, wl["cell"], wl["steps"] if steps is None else steps,
                                  wl["dt"], wl["seed"] + 1000 + seed_offset,
                                  trans_noise_frac=wl["trans_noise_frac"],
                                  rot_sigma=wl["rot_sigma"])


def make_sessions(wl: dict, steps: int):
    """The sessions of a multi-session workload: map, odometry stream (steps increments) and
    ground-truth poses of each.  ``batch64``: one office plan per session.  ``serve256``:
    n_maps plans, sessions assigned to them round-robin."""
    if "n_maps" in wl:
        maps = session_mix(wl["seed"], wl["n_maps"], side=wl["side"], ks=wl["ks"], cell=wl["cell"])
        occs = [floorplan.office_map(m["seed"], size=m["H"], cell=wl["cell"]) for m in maps]
        rng = np.random.Generator(np.random.PCG64(wl["seed"] + 77))
        mix = []
        for s in range(wl["n_sessions"]):
            m = dict(maps[s % wl["n_maps"]])
            m["K"] = int(wl["ks"][int(rng.integers(len(wl["ks"])))])
            m["map"] = s % wl["n_maps"]
            mix.append(m)
    else:
        mix = session_mix(wl["seed"], wl["n_sessions"], side=wl["side"], ks=wl["ks"], cell=wl["cell"])
        occs = [floorplan.office_map(m["seed"], size=m["H"], cell=wl["cell"]) for m in mix]
        for i, m in enumerate(mix):
            m["map"] = i
    out = []
    for i, m in enumerate(mix):
        occ = occs[m["map"]]
        walk = trajectory.random_walk(occ, wl["cell"], steps, wl["dt"], wl["seed"] * 100000 + 31 * i + 5,
                                      trans_noise_frac=wl["trans_noise_frac"], rot_sigma=wl["rot_sigma"])
        out.append(dict(m, occ=occ, odom=np.asarray(walk.odom, np.float64), poses=walk.poses))
    return out


def session_mix(seed: int, n: int, side=(128, 1024), ks=(36, 48, 64, 72), cell=0.05):
    """Per-session (H, W, K, map seed) for the batched and served workloads: square maps with
    side log-uniform in `side` (rounded to a multiple of 8) and K drawn from `ks`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(n):
        side_ = int(round(math.exp(rng.uniform(math.log(side[0]), math.log(side[1]))) / 8)) * 8
        k = int(ks[int(rng.integers(len(ks)))])
        out.append(dict(H=side_, W=side_, K=k, cell=cell, seed=seed * 1000 + s))
    return out
