"""Small fixed workload for profiler captures of the step kernels.

Runs ``--steps`` single-step launches of one model on a ``--size``^2 spinodal
lattice (FP32, the benchmark's parameters) through the C ABI, then synchronises.
Meant to be run under ``ncu -k regex:<model>_step -s <skip> -c <count>``.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--model", choices=["pp", "fe"], default="pp")
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--A", type=float, default=0.0, help="free-energy A != 0 runs the full-model kernel")
    args = ap.parse_args()
    import torch

    from paper_2403_11167_gb300 import build, inputs, lbm

    build.build()
    model = lbm.LBM_PSEUDOPOTENTIAL if args.model == "pp" else lbm.LBM_FREE_ENERGY
    p = lbm.lbm_params_default(model, precision=lbm.LBM_F32, a=0.25, Tr=0.85, tau_nu=0.8, A=args.A)
    ctx = lbm.Context(p, args.size, args.size)
    _, th = ctx.derived()
    ctx.set_density(inputs.spinodal_noise(args.size, args.size, 0.5 * (th.rho_l + th.rho_v), 0.01, seed=2403))
    for _ in range(args.steps):
        ctx.step(1)
    ctx.synchronize()
    torch.cuda.synchronize()
    print("profile case done:", args.model, args.size, args.steps)
    ctx.close()


if __name__ == "__main__":
    main()
