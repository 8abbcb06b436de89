"""Iteration counts n10 of the coarsening strategies and under a scaled penalty.

    python -m paper_1910_01900_gb300.strategies [--m 8] [--kmax 8] [--curved 0 1]
        [--orders cph chp cp phc hpc] [--pseq 0 1 2] [--penalty 1 10 100 1000]
        [--precision 1] [--markdown FILE]

The robustness studies of Section 4 on the cube: an m^3 mesh (Cartesian, or the
curved mapping with amplitude 0.1), degrees 1..kmax, Chebyshev(5,5), the
manufactured right-hand side (u = sin(pi x) sin(pi y) sin(pi z)), FCG from a
zero start to a relative residual of 1e-10.  n10 = -10 / log10(rho) with rho
the mean residual reduction per iteration.

Part 1: every order of the c, p and h steps in --orders (each must contain c
and p: the coarse solve works on degree-1 FE) with each p-sequence of the FE
and DG levels (0: floor(p/2), 1: p - 1, 2: straight to 1).  h halves the mesh
while m/2 >= 3 (8^3 -> 4^3).  Part 2: cph and phc with floor(p/2) and the
interior penalty factor scaled by each value of --penalty.

Prints one JSON line per solve; with --markdown, also writes the tables.
"""
import argparse
import json
import math


def n10_of(ctx, b, x, maxit):
    x.zero_()
    info = ctx.solve(b, x, rtol=1e-10, maxit=maxit, allow_notconv=True)
    return info.n10 if info.converged else math.inf, info.iterations, bool(info.converged)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=8)
    ap.add_argument("--kmax", type=int, default=8)
    ap.add_argument("--curved", type=int, nargs="+", default=[0, 1])
    ap.add_argument("--orders", nargs="+", default=["cph", "chp", "cp", "phc", "hpc"])
    ap.add_argument("--pseq", type=int, nargs="+", default=[0, 1, 2])
    ap.add_argument("--penalty", type=float, nargs="+", default=[1.0, 10.0, 100.0, 1000.0])
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--maxit", type=int, default=250)
    ap.add_argument("--markdown", default=None)
    args = ap.parse_args(argv)
    import torch

    from . import Context
    s = torch.cuda.Stream()
    rows = []
    ks = list(range(1, args.kmax + 1))

    def run(curved, k, order, pseq, pf, part):
        with torch.cuda.stream(s):
            ctx = Context(args.m, k, deform=curved, precision=args.precision, stream=s, coarsening=order,
                          p_coarsen=pseq, penalty_factor=pf)
            b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device="cuda")
            ctx.rhs(b)
            x = torch.zeros_like(b)
            n10, it, conv = n10_of(ctx, b, x, args.maxit)
            nl = ctx.num_levels
            ctx.close()
        r = {"part": part, "m": args.m, "curved": curved, "k": k, "order": order, "pseq": pseq,
             "penalty_factor": pf, "precision": args.precision, "levels": nl, "iterations": it,
             "converged": conv, "n10": None if math.isinf(n10) else round(n10, 2)}
        print(json.dumps(r), flush=True)
        rows.append(r)

    for curved in args.curved:
        for pseq in args.pseq:
            for order in args.orders:
                for k in ks:
                    run(curved, k, order, pseq, 1.0, "orders")
    for order in ("cph", "phc"):
        for pf in args.penalty:
            for k in ks:
                run(0, k, order, 0, pf, "penalty")

    if args.markdown:
        seqname = {0: "floor(p/2)", 1: "p-1", 2: "1"}
        out = []
        head = "| | " + " | ".join(str(k) for k in ks) + " |\n|---|" + "---|" * len(ks)

        def cell(r):
            return "-" if r is None or r["n10"] is None else f"{r['n10']:.1f}"

        def find(**kw):
            for r in rows:
                if all(r[a] == v for a, v in kw.items()):
                    return r
            return None
        for curved in args.curved:
            for pseq in args.pseq:
                out.append(f"\n{'Curved' if curved else 'Cartesian'} {args.m}^3, p-sequence {seqname[pseq]}: "
                           f"n10 by degree p\n\n{head}")
                for order in args.orders:
                    out.append(f"| {order} | " + " | ".join(cell(find(part="orders", curved=curved, pseq=pseq,
                                                                   order=order, k=k)) for k in ks) + " |")
        for order in ("cph", "phc"):
            out.append(f"\nPenalty factor scaled, {order}, floor(p/2), Cartesian {args.m}^3: n10 by degree p\n\n"
                       + head.replace("| |", "| factor |", 1))
            for pf in args.penalty:
                out.append(f"| {pf:g} | " + " | ".join(cell(find(part="penalty", order=order, penalty_factor=pf,
                                                               k=k)) for k in ks) + " |")
        with open(args.markdown, "w") as f:
            f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
