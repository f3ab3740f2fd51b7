"""Workload definitions (sizes and geometry only) for the measured configurations.

Each entry names a workload by what it is.  ``seed`` follows seed = 1000*index + mock.
"""
from __future__ import annotations

WORKLOADS = {
    # Plain FP64 Yamamoto P0,P2,P4 on a 64^3 CIC mesh, survey geometry, unit weights.
    "p024_fp64_64": dict(
        kind="power", n=64, box=1000.0, distance=1500.0, assign=2, interlace=0, n_gal=50_000,
        n_ran=500_000, n_gen=64, fkp_p0=None, kmin=0.0, dk=0.01, nbins=20, ells=(0, 2, 4),
        modified=(), precision="fp64", seed=0,
    ),
    # Yamamoto P0,P2,P4 + modified P4b,P6b,P8b, 512^3 TSC interlaced, FKP weights, mixed precision.
    "p024b_mixed_512": dict(
        kind="power", n=512, box=2000.0, distance=2500.0, assign=3, interlace=1, n_gal=2_000_000,
        n_ran=20_000_000, n_gen=256, fkp_p0=1.0e4, kmin=0.0, dk=0.01, nbins=80, ells=(0, 2, 4),
        modified=(4, 6, 8), precision="mixed", seed=1000,
    ),
    # The 512^3 power workload scaled to 256^3 (1/8 of the objects, same box): profiling size.
    "p024b_mixed_256": dict(
        kind="power", n=256, box=2000.0, distance=2500.0, assign=3, interlace=1, n_gal=250_000,
        n_ran=2_500_000, n_gen=128, fkp_p0=1.0e4, kmin=0.0, dk=0.01, nbins=40, ells=(0, 2, 4),
        modified=(4, 6, 8), precision="mixed", seed=1000,
    ),
    # Scoccimarro B0,B2 + compressed B_000, B_202 with analytic shot noise, periodic 256^3 TSC.
    "bispec_256": dict(
        kind="bispec", n=256, box=1000.0, assign=3, interlace=1, n_gal=1_000_000, n_gen=256,
        kmin=0.01, dk=0.01, nbins=19, scoc_ells=(0, 2), tripo_ells=(0, 2), precision="mixed",
        seed=2000,
    ),
    # 96 survey mocks of uneven size in one batch: 32 each on 128^3, 192^3 and 256^3 meshes, box side
    # L ~ U[500, 1500], N_g log-uniform in [1e5, 2e6], N_r = 10 N_g, box centre at 1.5 L; P_0,2,4 on
    # bins of 0.01 up to k_N, B_0 on 19 bins from 0.01 truncated at k_N/2.
    "batch_96": dict(
        kind="batch", sizes=(128, 192, 256), per_size=32, box_range=(500.0, 1500.0),
        n_gal_range=(1e5, 2e6), ran_factor=10, distance_factor=1.5, assign=3, interlace=1,
        fkp_p0=1.0e4, dk=0.01, pk_nbins_max=80, bk_kmin=0.01, bk_nbins=19, ells=(0, 2, 4),
        precision="mixed", seed=3000,
    ),
    # Gradients of P_0,2,4 (global LOS) and of the equilateral B_0 (19 bins) with respect to the
    # mesh and, through the TSC adjoint, the galaxy positions: periodic 1024^3, 1e7 galaxies.
    "adjoint_1024": dict(
        kind="adjoint", n=1024, box=3000.0, assign=3, interlace=0, n_gal=10_000_000, n_gen=256,
        kmin=0.01, dk=0.01, nbins=19, ells=(0, 2, 4), b0=True, precision="mixed", seed=4000,
    ),
    # The same at 32^3 for finite-difference checks (box scaled to keep k_N, 1/32 of the side).
    "adjoint_32": dict(
        kind="adjoint", n=32, box=93.75, assign=3, interlace=0, n_gal=2_000, n_gen=32,
        kmin=0.1, dk=0.1, nbins=4, ells=(0, 2, 4), b0=True, precision="fp64", seed=4001,
    ),
}


def workload(name):
    return dict(WORKLOADS[name])
