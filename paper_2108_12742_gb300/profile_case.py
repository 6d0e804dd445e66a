"""Launches one sweep kernel of a chosen workload size, for profiler captures.

    python -m paper_2108_12742_gb300.profile_case --n 2048 --precision fp32 --dir 0 --nrep 2

Builds the 2D four-quadrant Euler workload (the benchmark's, at n x n cells;
``--ndim 3`` uses the 3D periodic blast workload at n^3; ``--workload
riemann2`` the 2D Riemann configuration 2 of Sec. 4.3 on [-1, 1]^2), sets the
re-decision mode of FP32 bulk (``--redecide in_sweep|grid``), the tiles
(``--ta/--ts``, default: the library's defaults) and launches the sweep
kernel of axis ``--dir`` nrep times through ``enoao_time_sweep``, printing the
mean launch time.  The device holds three state buffers and one
right-hand-side buffer of the chosen size.  ``--steps-before K`` first takes
K Runge-Kutta steps, so the launches see evolved rather than initial data.
"""
from __future__ import annotations

import argparse

import paper_2108_12742_gb300 as eno
from paper_2108_12742_gb300 import inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--ndim", type=int, default=2, choices=[2, 3])
    ap.add_argument("--order", type=int, default=5)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--dir", type=int, default=0)
    ap.add_argument("--nrep", type=int, default=2)
    ap.add_argument("--ta", type=int, default=0)
    ap.add_argument("--ts", type=int, default=0)
    ap.add_argument("--steps-before", type=int, default=0,
                    help="Runge-Kutta steps taken before the timed launches (evolved data)")
    ap.add_argument("--workload", default="quadrants", choices=["quadrants", "riemann2"])
    ap.add_argument("--redecide", default="in_sweep", choices=["in_sweep", "grid"])
    args = ap.parse_args()
    n = args.n
    prec = eno.FP32_BULK if args.precision == "fp32" else eno.FP64
    if args.workload == "riemann2":
        U = inputs.riemann2d(2, n, n)
        s = eno.Solver((n, n), (-1.0, -1.0), (1.0, 1.0), system=eno.EULER, order=args.order,
                       bc=eno.TRANSMISSIVE, precision=prec)
    elif args.ndim == 2:
        U = inputs.euler2d_quadrants(n, n, seed=1)
        s = eno.Solver((n, n), (0.0, 0.0), (1.0, 1.0), system=eno.EULER, order=args.order,
                       bc=eno.TRANSMISSIVE, precision=prec)
    else:
        U = inputs.euler3d_blast(n, seed=1)
        s = eno.Solver((n, n, n), (0.0,) * 3, (1.0,) * 3, system=eno.EULER, order=args.order,
                       bc=eno.PERIODIC, precision=prec)
    with s:
        s.set_redecide(eno.REDECIDE_GRID if args.redecide == "grid" else eno.REDECIDE_IN_SWEEP)
        s.init_state(U)
        if args.steps_before:
            s.advance_steps(args.steps_before, 0.5)
        if args.ta or args.ts:
            s.set_tiles(args.dir, args.ta, args.ts)
        ms = s.time_sweep(args.dir, args.nrep)
        print(f"sweep axis {args.dir} {args.precision} n={n} tiles={s.get_tiles(args.dir)}: "
              f"{ms:.3f} ms per launch")


if __name__ == "__main__":
    main()
