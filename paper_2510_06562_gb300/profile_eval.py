"""Repeated force evaluations of one model on a synthetic system, for kernel
profilers (no timing, no output besides a one-line summary).

    python -m paper_2510_06562_gb300.profile_eval --precision bf16 --which big --evals 3
    python -m paper_2510_06562_gb300.profile_eval --precision bf16 --respa 6 --evals 1
    python -m paper_2510_06562_gb300.profile_eval --precision bf16 --respa 4 --dt 6 --n-inner 6 --evals 0
    python -m paper_2510_06562_gb300.profile_eval --precision bf16 --distill 4 --evals 0
"""
from __future__ import annotations

import argparse

import numpy as np

from . import dmts as D
from . import inputs as I


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--which", default="big", choices=["small", "big"])
    ap.add_argument("--system", default="water12288", choices=["water192", "water12288"])
    ap.add_argument("--evals", type=int, default=3)
    ap.add_argument("--respa", type=int, default=0, help="first: this many outer steps of Algorithm 1")
    ap.add_argument("--dt", type=float, default=3.0, help="outer step of --respa (fs)")
    ap.add_argument("--n-inner", type=int, default=3, help="inner steps per outer step of --respa")
    ap.add_argument("--distill", type=int, default=0,
                    help="then: two energy + force distillation gradients over this many frames (the structure "
                         "plus seeded 0.02 A displacements, seeded reference forces and energies)")
    ap.add_argument("--options", default=None, help="context options (JSON)")
    args = ap.parse_args()
    s = I.water_12288(0) if args.system == "water12288" else I.water_192(0)
    prec = D.BF16_MLP if args.precision == "bf16" else D.FP32
    sa, ba = I.small_arch(s.n_species), I.big_arch(s.n_species)
    with D.Context(s, ba, I.init_params(ba, 3), sa, I.init_params(sa, 2), precision=prec,
                   options=args.options) as ctx:
        ctx.set_state(s.x)
        which = D.BIG if args.which == "big" else D.SMALL
        if args.respa:
            ctx.respa_step(args.respa, args.dt, args.n_inner, energies=False)
        E, F = np.zeros(1), np.zeros((1, 3))
        for _ in range(args.evals):
            E, F = ctx.forces(which)
        if args.distill:
            rng = np.random.default_rng(0)
            frames = np.stack([s.x + rng.normal(scale=0.02, size=s.x.shape) for _ in range(args.distill)])
            frames -= s.box[0] * np.floor(frames / s.box[0])
            f_ref = rng.normal(scale=0.5, size=frames.shape)
            e_ref = np.full(args.distill, 0.75 * s.n_atoms)
            for _ in range(2):
                loss, _ = ctx.distill_grad(frames, f_ref, e_ref, 1.0)
            print(f"distillation loss {loss:.6f} over {args.distill} frames")
    print(f"{args.system} {args.which} {args.precision}: E={E[0]:.6f} eV, rms F={np.sqrt(np.mean(F ** 2)):.4f} eV/A")


if __name__ == "__main__":
    main()
