"""Command-line runner: quench one lattice, one asynchronous multispin ensemble
or the batched workload for a number of sweeps and print energies as JSON.

    python -m paper_1411_0127_gb300 sweep --L 1024 --T 0.9 --kind mt19937 --sweeps 10
    python -m paper_1411_0127_gb300 amsc  --L 512  --T 0.9 --kind mt19937 --sweeps 3
    python -m paper_1411_0127_gb300 batch --kind mt19937 --config 0,32,1,1 --sweeps 128 --group 64

`sweep` runs isg_create2 + isg_sweep; `amsc` runs isg_amsc_create + isg_amsc_sweep
with the 32 systems' seeds of workloads.amsc_seeds(L); `batch` runs
isg_batch_create + isg_batch_run on the 512 samples of workloads.batch_samples()
(--L and --T are then ignored) with the execution configuration --config
(shape, capacity, resident, words per lane; "auto": the autotuner) in launches of
--group sweeps.  --every prints the energies every that many sweeps (0: at the
end only)."""
import argparse
import json
import sys
import time


def main(argv=None) -> int:
    p = argparse.ArgumentParser(prog="python -m paper_1411_0127_gb300")
    p.add_argument("mode", choices=["sweep", "amsc", "batch"])
    p.add_argument("--L", type=int, default=64)
    p.add_argument("--T", type=float, default=0.9, help="temperature (beta = 1/T)")
    p.add_argument("--kind", default="mt19937", help="minstd or mt19937")
    p.add_argument("--sweeps", type=int, default=10)
    p.add_argument("--every", type=int, default=0)
    p.add_argument("--seed-J", type=int, default=1)
    p.add_argument("--seed-spin", type=int, default=2)
    p.add_argument("--seed-rng", type=int, default=None)
    p.add_argument("--config", default="0,32,1,1", help="batch: shape,capacity,resident,words_per_lane or auto")
    p.add_argument("--group", type=int, default=64, help="batch: sweeps per persistent launch")
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
    elif a.mode == "batch":
        sm = workloads.batch_samples()
        b = isg.Batch([x.L for x in sm], [x.seed_J for x in sm], [v for x in sm for v in x.seed_spin],
                      [1.0 / x.T for x in sm], a.kind)
        if a.config == "auto":
            b.autotune()
        else:
            b.set_config(*[int(v) for v in a.config.split(",")])

        class _Runner:                    # sweep(n) in launches of --group sweeps
            def sweep(self, n):
                b.run(n, a.group)

            def close(self):
                b.close()

        h = _Runner()

        def measure():
            E, Q = b.measure()
            return {"config": list(b.get_config()), "E_sum": int(E.sum()), "Q_sum": int(Q.sum())}
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
            L = "mixed" if a.mode == "batch" else a.L
            print(json.dumps({"mode": a.mode, "L": L, "sweeps": done, **measure()}), flush=True)
    torch.cuda.synchronize()
    print(json.dumps({"mode": a.mode, "wall_s": time.perf_counter() - t0}), flush=True)
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
