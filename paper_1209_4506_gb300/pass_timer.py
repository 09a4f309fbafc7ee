"""Time the compiled variants of one pass kind on a grid, or run one variant alone (for a profiler).

    python -m paper_1209_4506_gb300.pass_timer --shape 512,512,512            # every a and b variant
    python -m paper_1209_4506_gb300.pass_timer --shape 512,128,512 --only 2:13  # variant 13 of the a pass, 3 launches
    python -m paper_1209_4506_gb300.pass_timer --splat cfg5                     # fused vs separate splat + r2c
    python -m paper_1209_4506_gb300.pass_timer --splat cfg5 --only fused        # the fused pass alone, 3 launches

Pass kinds follow hartree_plan_set_variants: 0 the c passes, 1 the b passes (forward and inverse
timed with the same pick), 2 the a pass.  The density is white noise; the grid's half spectrum
stays in the plan's workspace between launches, as in a solve.  CUDA-event times on the current
stream, after three warm-up launches.
"""
import argparse

import torch

from . import capi, synth
from .hartree import HartreePlan, atoms_reorder

PASS_OF_KIND = {0: (0, 4), 1: (1, 3), 2: (2,)}


def _time(fn, reps, stream):
    for _ in range(3):
        fn()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps * 1000.0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--shape", default="512,512,512")
    ap.add_argument("--cell", default="50,50,50")
    ap.add_argument("--kinds", default="2,1", help="pass kinds to sweep")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--only", default=None, help="kind:variant -> three launches of that variant alone")
    ap.add_argument("--splat", default=None, choices=["cfg5", "cfg3a"],
                    help="atoms of a synthetic system: the splat fused into pass 0 against the splat and pass 0")
    args = ap.parse_args(argv)
    if args.splat:
        return splat_main(args)
    shape = tuple(int(x) for x in args.shape.split(","))
    cell = tuple(float(x) for x in args.cell.split(","))
    plan = HartreePlan(shape, cell, 0.5, "fp32")
    rho = torch.randn(shape, device="cuda")
    vh = torch.empty_like(rho)
    plan.solve_density(rho, vh)
    torch.cuda.synchronize()
    if args.only:
        kind, var = (int(x) for x in args.only.split(":"))
        choice = [0, 0, 0]
        choice[kind] = var
        plan.set_variants(choice)
        for _ in range(3):
            for p in PASS_OF_KIND[kind]:
                plan.solve_pass(p, rho=rho, vh=vh)
        torch.cuda.synchronize()
        plan.device_status()
        print("ok")
        return
    stream = torch.cuda.current_stream()
    for kind in (int(k) for k in args.kinds.split(",")):
        total = 0  # picks of this kind: V variants, or V * V picks for the pairs of c and b passes
        while True:
            choice = [0, 0, 0]
            choice[kind] = total
            try:
                plan.set_variants(choice)
            except capi.HartreeError:
                break
            total += 1
        singles = total if kind == 2 else int(round(total ** 0.5))
        for var in range(singles):
            choice = [0, 0, 0]
            choice[kind] = var
            plan.set_variants(choice)
            times = [_time(lambda p=p: plan.solve_pass(p, rho=rho, vh=vh), args.reps, stream)
                     for p in PASS_OF_KIND[kind]]
            print(f"kind {kind} variant {var}: " + ", ".join(f"pass {p} {t:.1f} us"
                                                          for p, t in zip(PASS_OF_KIND[kind], times)), flush=True)
    plan.device_status()
    plan.close()


def splat_main(args):
    S = {"cfg5": synth.config5, "cfg3a": synth.config3a}[args.splat]()
    apl = 16
    perm, _ = atoms_reorder(S.pos, (S.n_atoms + apl - 1) // apl)
    pos = torch.tensor(S.pos[perm], device="cuda")
    q = torch.tensor(S.q[perm], device="cuda")
    fused = HartreePlan(S.n, S.cell, S.sigma, "fp32", atoms_per_leaf=apl, max_atoms=S.n_atoms,
                        flags=capi.HARTREE_FLAG_FUSED_SPLAT)
    if args.only == "fused":
        for _ in range(3):
            fused.splat_pass(pos, q)
        torch.cuda.synchronize()
        fused.device_status()
        print("ok")
        return
    plain = HartreePlan(S.n, S.cell, S.sigma, "fp32", atoms_per_leaf=apl, max_atoms=S.n_atoms)
    rho = torch.empty(S.n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def separate():
        plain.splat(pos, q, rho)
        plain.solve_pass(0, rho=rho)

    t_f = _time(lambda: fused.splat_pass(pos, q), args.reps, stream)
    t_s = _time(separate, args.reps, stream)
    print(f"{args.splat}: fused splat + pass 0 {t_f:.1f} us, splat + pass 0 {t_s:.1f} us")
    fused.close()
    plain.close()


if __name__ == "__main__":
    main()
