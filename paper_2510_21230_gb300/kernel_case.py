"""Run one force evaluation configuration a few times on a synthetic workload
and print its CUDA-event time per evaluation -- a small driver for profilers
(it launches only the cell build, LJ and the chosen ATM or surrogate kernel).

    python -m paper_2510_21230_gb300.kernel_case --workload liquid_n256k \\
        --trav 3c08 --trunc pair --prec fp32c --reps 3

With --prec surrogate the model is random (seeded) with the descriptor
normalisation of the workload's own descriptors.  --n N replaces the workload
by a liquid of N molecules at rho 0.8 (fcc start, seed 7000); N = 104052
gives the cell edge of the 256,000-molecule liquid (20 instead of 27 cells per
axis).  The ATM kernel's own time comes from the library's launch profiler.
"""
import argparse
import os
import sys

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2510_21230_gb300 import atm3, build, synth  # noqa: E402


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="liquid_n32k", choices=sorted(synth.CONFIGS))
    p.add_argument("--trav", default="3c08", choices=sorted(atm3.TRAVERSALS))
    p.add_argument("--trunc", default="pair", choices=sorted(atm3.TRUNCATIONS))
    p.add_argument("--prec", default="fp32c", choices=sorted(atm3.PRECISIONS))
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--n", type=int, default=0)
    p.add_argument("--nwarps", type=int, default=0)
    a = p.parse_args()
    import torch
    build.build()
    cfg = synth.homogeneous(a.n, 0.8, 1.0, seed=7000) if a.n > 0 else synth.config(a.workload)
    name = "liquid_n%d" % a.n if a.n > 0 else a.workload
    stream = torch.cuda.current_stream()
    with atm3.AtmSystem(cfg["box"], cfg["n"], rc=2.5, nu=0.073, stream=stream.cuda_stream) as s:
        s.set_state(cfg["x"], cfg["v"])
        s.build_cells()
        if a.prec == "surrogate":
            D, _ = s.surrogate_descriptors()
            sd = D.std(axis=0)
            s.surrogate_set_model(synth.sur_params(7), D.mean(axis=0),
                                  np.where(sd > 1e-12, sd, 1.0).astype(np.float32))
        if a.nwarps:
            s.set_options(nwarps=a.nwarps)
        s.compute_forces(a.trav, a.trunc, a.prec)
        torch.cuda.synchronize()
        s.set_profiling(True)
        times = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(a.reps):
                s.compute_forces(a.trav, a.trunc, a.prec, sync=False)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / a.reps)
        r = s.results()[0]
        prof = s.get_profile()
    atm = prof["ms_atm"] / max(1, prof["n_atm_launches"])
    print("%s %s %s %s: %.4f ms per evaluation (median of 3 x %d; cells excluded), ATM kernel "
          "%.4f ms, n_int3 %d" % (name, a.trav, a.trunc, a.prec, sorted(times)[1], a.reps, atm,
                                  r["n_int3"]))


if __name__ == "__main__":
    main()
