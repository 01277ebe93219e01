"""Command-line runner: quench one lattice or one asynchronous multispin
ensemble for a number of sweeps and print its energies as JSON.

    python -m paper_1411_0127_gb300 sweep --L 1024 --T 0.9 --kind mt19937 --sweeps 10
    python -m paper_1411_0127_gb300 amsc  --L 512  --T 0.9 --kind mt19937 --sweeps 3

`sweep` runs isg_create2 + isg_sweep; `amsc` runs isg_amsc_create + isg_amsc_sweep
with the 32 systems' seeds of workloads.amsc_seeds(L).  --every prints the
energies every that many sweeps (0: at the end only)."""
import argparse
import json
import sys
import time


def main(argv=None) -> int:
    p = argparse.ArgumentParser(prog="python -m paper_1411_0127_gb300")
    p.add_argument("mode", choices=["sweep", "amsc"])
    p.add_argument("--L", type=int, default=64)
    p.add_argument("--T", type=float, default=0.9, help="temperature (beta = 1/T)")
    p.add_argument("--kind", default="mt19937", help="minstd or mt19937")
    p.add_argument("--sweeps", type=int, default=10)
    p.add_argument("--every", type=int, default=0)
    p.add_argument("--seed-J", type=int, default=1)
    p.add_argument("--seed-spin", type=int, default=2)
    p.add_argument("--seed-rng", type=int, default=None)
    a = p.parse_args(argv)

    import torch
    import paper_1411_0127_gb300 as isg
    from paper_1411_0127_gb300 import workloads

    if not torch.cuda.is_available():
        print("a CUDA device is required", file=sys.stderr)
        return 2
    beta = 1.0 / a.T
    if a.mode == "sweep":
        h = isg.Sim(a.L, a.seed_J, a.seed_spin, beta, a.kind, seed_rng=a.seed_rng)
        measure = lambda: {"E": h.energy(), "hash": h.hash()}
    else:
        J, S = workloads.amsc_seeds(a.L)
        h = isg.Amsc(a.L, J, S, a.seed_rng if a.seed_rng is not None else 12345, beta, a.kind)
        measure = lambda: {"E": h.energies().tolist()}
    step = a.every if a.every > 0 else a.sweeps
    done = 0
    t0 = time.perf_counter()
    while done < a.sweeps:
        n = min(step, a.sweeps - done)
        h.sweep(n)
        done += n
        if a.every > 0 or done == a.sweeps:
            torch.cuda.synchronize()
            print(json.dumps({"mode": a.mode, "L": a.L, "sweeps": done, **measure()}), flush=True)
    torch.cuda.synchronize()
    print(json.dumps({"mode": a.mode, "wall_s": time.perf_counter() - t0}), flush=True)
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
