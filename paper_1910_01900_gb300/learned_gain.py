"""What one V-cycle leaves with the learned post-smoother, without it, and with Chebyshev.

    python -m paper_1910_01900_gb300.learned_gain

Two cases: 8^3 Cartesian k = 3 with an FP64 cycle (40,000 pairs, 30 epochs, seed
7: the GPU test's case) and 32^3 curved k = 4 with an FP32 cycle (100,000
pairs, 20 epochs, seed 2024: the learned-smoother workload).  After training,
one V-cycle z = M r is applied to a seeded uniform r (seed 71) with
  no_post    Chebyshev pre-smoothing, no post-smoothing on the finest level
             (the cycle without the network),
  net_post   the same plus one network post-step (the default learned cycle),
  net_2_2    two network steps before and after the coarse correction,
  chebyshev  Chebyshev(5,5), the plain cycle,
and reports what is left: the residual ||r - A z|| / ||r||, and the error
against x* = A^-1 r (flexible CG with the plain cycle to 1e-12) in the energy
norm ||x* - z||_A / ||x*||_A and in the 2-norm.  One JSON line per case.
"""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import sipg_inputs  # noqa: E402  (seeded input generators)

CASES = [(8, 3, 0, 0, 40000, 30, 7), (32, 4, 1, 1, 100000, 20, 2024)]
CYCLES = (("no_post", (1, 0, 0)), ("net_post", (1, 0, 1)), ("net_2_2", (1, 2, 2)), ("chebyshev", (0,)))


def measure(m, k, curved, precision, npairs, epochs, seed):
    import torch

    from . import Context
    ctx = Context(m, k, deform=curved, precision=precision)
    info = ctx.train_smoother(npairs=npairs, epochs=epochs, seed=seed)
    r = torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(), 71)).cuda()
    xs = torch.zeros_like(r)
    ctx.set_smoother(0)
    ctx.solve(r, xs, rtol=1e-12, maxit=200)

    def energy(e):
        ae = torch.empty_like(e)
        ctx.apply(e, ae)
        return torch.dot(e, ae).item() ** 0.5
    e0 = energy(xs)
    out = {"m": m, "k": k, "curved": curved, "precision": precision, "pairs": npairs, "epochs": epochs,
           "step_reduction": info.step_reduction, "damping": info.damping}
    for name, cfg in CYCLES:
        ctx.set_smoother(*cfg)
        z, az = torch.empty_like(r), torch.empty_like(r)
        ctx.vcycle(r, z)
        ctx.apply(z, az)
        out[name] = {"residual_left": (torch.linalg.norm(r - az) / torch.linalg.norm(r)).item(),
                     "energy_error_left": energy(xs - z) / e0,
                     "l2_error_left": (torch.linalg.norm(xs - z) / torch.linalg.norm(xs)).item()}
    ctx.close()
    return out


def main():
    for case in CASES:
        print(json.dumps(measure(*case)), flush=True)


if __name__ == "__main__":
    main()
