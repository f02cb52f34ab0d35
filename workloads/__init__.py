"""Seeded synthetic workloads for the CIL hot path (arXiv 2203.14742).

This module holds the *inputs* only: workload sizes, parameter draws and
synthetic pattern sets.  It contains none of the method's arithmetic (no
stepping, no distances, no statistics), so both the oracle and the CUDA path
may use it.  Random numbers the method itself draws (initial noise, bootstrap
indices) are NOT made here: each side evaluates the same published
counter-based generator (SplitMix64) from a seed given here.

The paper simulates its training data at theta_0 (Table 1), so simulated
patterns are the paper's workload; there is no dataset to stand in for.

Workloads (sizes follow the paper's Table 1 models and the hot-path configs):
  c1  FHN 32x32, 2 sets x 16, dt 2^-8, 2000 steps, both species (d = 2048),
      M = 8 radii, b = 1.3, 50 resamples, noise U(-0.05, 0.05).
  c2  FHN 64x64, 2 sets x 64, dt 2^-10, 10^4 steps, u only (d = 4096),
      M = 16, 200 resamples.
  c3  GM 128x128, rho = 1, mu = 0.5 +-10 %, 2 sets x 256, dt 2^-10,
      2*10^4 steps, both species (d = 32768), M = 16, noise U(0, 0.01).
  c4  64 parameter vectors x 128 realisations: 16 FHN + 16 GM at 64x64
      (10^4 steps), 16 FHN + 16 GM at 128x128 (2*10^4 steps); per vector
      2 sets x 64, 200 resamples, M = 16.  dt is the largest power of two
      below the explicit diffusion limit h^2/(4 D_max): FHN 2^-10 (64^2),
      2^-12 (128^2); GM 2^-8 (64^2), 2^-10 (128^2).
  c5  FHN 64x64, 32 realisations (2 x 16), dt 2^-10, 5000 steps, M = 16,
      smoothed CIL with tau_k = 0.05 R_k, cotangent 1/M.
  c6  Brusselator ("BZ", Table 1) 64x64, 2 sets x 64, dt 2^-8, 25600 steps
      (T = 100), both species (d = 8192), noise U(0, 0.01), M = 16.
  c7  reaction-diffusion-ODE model (Sec. 4.3, Table 1 "RD"), 64 nodes, 2 sets
      x 100 realisations (the 100 model runs per cost evaluation of Sec. 5),
      t in [0, 50] by the adaptive stabilised RK2 (rtol = atol = 1e-6),
      initial u = U(0, 2) noise smoothed by 10 moving-average passes, w = 0;
      (m1, m2) within +-5 % of (1.44, 4.1); both species (d = 128), M = 13.
  c8  synthetic CIL with bootstrapping (Alg. 6) in Table 1's setting: FHN
      64x64 to T = 100 (102400 Euler steps of 2^-10), N_syn = 1000 model
      runs at theta (Sec. 5: 1000 runs per cost evaluation), N_set = 50,
      the six features on both species, M = 13 radii per feature with the
      power law fitted to the range, n_CIL = 1000 resamples; the data set is
      50 patterns simulated at theta_0 (seed + 1000).
  glarge  the paper's SCIL scale (N_syn = 1000, Sec. 5.3): 2 sets x 1024
      patterns of d = 32768 for the Gram kernel alone.
"""
import math

import numpy as np

FHN, GM, DIFF, BZ, RDODE = 0, 1, 2, 3, 4

SEED_BASE = 0x2203147420000000

# Table 1 values (theta_0 and the diffusion coefficients), in this package's
# species order (u, v); see the model mapping in oracle/rd.c.
FHN_THETA0 = (2.8e-4, 0.05, 10.0, 1.0)      # Du = nu_2, Dv = nu_1, eps, a = alpha
GM_THETA0 = (2.5e-4, 0.01, 1.0, 0.5)        # Du = nu_1, Dv = nu_2, rho, mu = mu_v
BZ_THETA0 = (1.6e-3, 1.32e-2, 4.5, 6.96)    # Brusselator: Du = nu_1, Dv = nu_2, A, B
# 1-D reaction-diffusion-ODE model (Sec. 4.3): (unused, D, m1, m2, m3, k)
RDODE_THETA0 = (0.0, 1.0, 1.44, 4.1, 4.1, 0.01)


def seed_of(cfg_index: int) -> int:
    return SEED_BASE + cfg_index


def draw_params(model: int, seed: int, n: int = 1):
    """n parameter vectors, each uniform in a box around theta_0.

    FHN: Du, Dv, eps within +-10 % of Table 1; a in [0.9, 1.0] (a < 1 makes
    the equilibrium strictly stable to homogeneous perturbations).
    GM:  mu within +-10 % of 0.5; rho = 1; Table 1 diffusions.
    BZ:  A in [4.3, 4.6], B in [6.9, 7.2] around Table 1's (4.5, 6.96);
         Table 1 diffusions.
    RDODE: m1, m2 within +-5 % of Table 1's (1.44, 4.1); D, m3, k fixed.
    The oracle test suite checks every drawn vector for a diffusion-driven
    instability on the discrete grid.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        if model == FHN:
            Du = FHN_THETA0[0] * rng.uniform(0.9, 1.1)
            Dv = FHN_THETA0[1] * rng.uniform(0.9, 1.1)
            eps = FHN_THETA0[2] * rng.uniform(0.9, 1.1)
            a = rng.uniform(0.9, 1.0)
            out.append((Du, Dv, eps, a))
        elif model == GM:
            mu = GM_THETA0[3] * rng.uniform(0.9, 1.1)
            out.append((GM_THETA0[0], GM_THETA0[1], 1.0, mu))
        elif model == BZ:
            # A in [4.3, 4.6], B in [6.9, 7.2]: above the Turing threshold
            # (1 + A sqrt(Du/Dv))^2 <= 6.77 and below the Hopf value 1 + A^2
            A = rng.uniform(4.3, 4.6)
            B = rng.uniform(6.9, 7.2)
            out.append((BZ_THETA0[0], BZ_THETA0[1], A, B))
        elif model == RDODE:
            m1 = RDODE_THETA0[2] * rng.uniform(0.95, 1.05)
            m2 = RDODE_THETA0[3] * rng.uniform(0.95, 1.05)
            out.append((0.0, RDODE_THETA0[1], m1, m2, RDODE_THETA0[4], RDODE_THETA0[5]))
        else:
            raise ValueError("model")
    return out


def group(model, G, n_real, params, dt, n_steps, noise, seed, species_mask):
    return {"model": model, "G": G, "n_real": n_real, "params": tuple(params),
            "dt": dt, "n_steps": n_steps, "noise": tuple(noise), "seed": seed,
            "species_mask": species_mask}


def config(name: str, steps_scale: float = 1.0):
    """Workload description.  steps_scale shortens the integration (tests)."""
    def steps(n):
        return max(1, int(round(n * steps_scale)))

    if name == "c1":
        s = seed_of(1)
        p = draw_params(FHN, s)[0]
        g = group(FHN, 32, 32, p, 2.0 ** -8, steps(2000), (-0.05, 0.05), s, 3)
        return {"name": name, "groups": [g], "n1": 16, "n2": 16, "M": 8, "b": 1.3,
                "T_res": 50, "seed": s}
    if name == "c2":
        s = seed_of(2)
        p = draw_params(FHN, s)[0]
        g = group(FHN, 64, 128, p, 2.0 ** -10, steps(10000), (-0.05, 0.05), s, 1)
        return {"name": name, "groups": [g], "n1": 64, "n2": 64, "M": 16, "b": 1.3,
                "T_res": 200, "seed": s}
    if name == "c3":
        s = seed_of(3)
        p = draw_params(GM, s)[0]
        g = group(GM, 128, 512, p, 2.0 ** -10, steps(20000), (0.0, 0.01), s, 3)
        return {"name": name, "groups": [g], "n1": 256, "n2": 256, "M": 16, "b": 1.3,
                "T_res": 200, "seed": s}
    if name == "c4":
        s = seed_of(4)
        groups = []
        k = 0
        for G, n_steps in ((64, 10000), (128, 20000)):
            for model in (FHN, GM):
                ps = draw_params(model, s + 17 * k, 16)
                for j, p in enumerate(ps):
                    if model == FHN:
                        # 128x128 FHN: h^2/(4 Dv) = 2.8e-4, so the power of two is 2^-12.
                        dt = 2.0 ** -10 if G == 64 else 2.0 ** -12
                        noise, mask = (-0.05, 0.05), (1 if G == 64 else 3)
                    else:
                        dt, noise, mask = (2.0 ** -8 if G == 64 else 2.0 ** -10), (0.0, 0.01), 3
                    groups.append(group(model, G, 128, p, dt, steps(n_steps), noise,
                                        s + 1000 * (k + 1) + j, mask))
                k += 1
        return {"name": name, "groups": groups, "n1": 64, "n2": 64, "M": 16, "b": 1.3,
                "T_res": 200, "seed": s}
    if name == "c6":
        s = seed_of(6)
        p = draw_params(BZ, s)[0]
        # Table 1: T = 100 on 64 x 64; h^2 / (4 Dv) = 4.8e-3, so dt = 2^-8
        g = group(BZ, 64, 128, p, 2.0 ** -8, steps(25600), (0.0, 0.01), s, 3)
        return {"name": name, "groups": [g], "n1": 64, "n2": 64, "M": 16, "b": 1.3,
                "T_res": 200, "seed": s}
    if name == "c7":
        s = seed_of(7)
        p = draw_params(RDODE, s)[0]
        # Table 1: t in [0, 50] on 64 nodes; dt * n_steps is only the horizon
        g = group(RDODE, 64, 200, p, 2.0 ** -10, steps(51200), (0.0, 2.0), s, 3)
        return {"name": name, "groups": [g], "n1": 100, "n2": 100, "M": 13, "b": 1.3,
                "T_res": 200, "seed": s, "rkc_tol": 1e-6}
    if name == "c8":
        s = seed_of(8)
        p = draw_params(FHN, s)[0]
        p0 = draw_params(FHN, s + 1000)[0]
        g = group(FHN, 64, 1000, p, 2.0 ** -10, steps(102400), (-0.05, 0.05), s, 3)
        gd = group(FHN, 64, 50, p0, 2.0 ** -10, steps(102400), (-0.05, 0.05), s + 1000, 3)
        return {"name": name, "groups": [g], "data_group": gd, "n_set": 50, "M": 13, "law": "fitted",
                "features": 63, "T_res": 1000, "seed": s}
    if name == "c5":
        s = seed_of(5)
        p = draw_params(FHN, s)[0]
        g = group(FHN, 64, 32, p, 2.0 ** -10, steps(5000), (-0.05, 0.05), s, 1)
        return {"name": name, "groups": [g], "n1": 16, "n2": 16, "M": 16, "b": 1.3,
                "tau_frac": 0.05, "seed": s}
    raise KeyError(name)


def cosine_patterns(n: int, G: int, n_species: int, seed: int, n_modes: int = 6,
                    amp: float = 1.0, offset: float = 0.0):
    """n synthetic pattern vectors [n, n_species*G*G] float32: each species a
    sum of n_modes random cosine modes cos(pi k (x+1/2)/G) cos(pi l (y+1/2)/G)
    with random k, l in [1, G/4] and N(0,1) amplitudes, scaled by amp and
    shifted by offset.  Stands in for stepped patterns where the stepper is
    not part of what is tested."""
    rng = np.random.default_rng(seed)
    xs = (np.arange(G) + 0.5) / G
    out = np.empty((n, n_species, G, G), np.float64)
    for i in range(n):
        for s in range(n_species):
            f = np.zeros((G, G))
            for _ in range(n_modes):
                k = rng.integers(1, max(2, G // 4) + 1)
                l = rng.integers(1, max(2, G // 4) + 1)
                f += rng.normal() * np.outer(np.cos(math.pi * l * xs), np.cos(math.pi * k * xs))
            out[i, s] = f
    out = out * (amp / max(1e-30, np.abs(out).max())) + offset
    return out.reshape(n, -1).astype(np.float32)


def clustered_patterns(n: int, d: int, seed: int, n_centres: int = 4, spread: float = 0.2):
    """n float32 vectors in R^d drawn around a few random centres, so that the
    cross-set distances spread over several radii bins."""
    rng = np.random.default_rng(seed)
    centres = rng.normal(size=(n_centres, d))
    which = rng.integers(0, n_centres, size=n)
    scale = rng.uniform(0.3, 1.0, size=(n, 1)) * spread
    X = centres[which] + scale * rng.normal(size=(n, d))
    return X.astype(np.float32)
