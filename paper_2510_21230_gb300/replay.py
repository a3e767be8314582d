"""Replay of the single-phase validation runs of section 5.1 (Table 1phase,
Fig. rdfs) on the library: both thermodynamic states run together as a batch
of two replicas on one GPU.

Protocol (the paper's, with the step counts as options):
  * cubic box of edge 12.5, r_c = 2.5, dt = 0.004, simple cubic start;
    state A: T = 1.033, rho = 0.65 (N = 1270); state B: T = 0.746,
    rho = 0.817 (N = 1596);
  * melting with LJ only (nu = 0), then an LJ-only production run (the
    nu = 0 reference), then, from its last configuration, a production run
    with LJ + ATM (nu = 0.072) for every traversal and truncation asked for;
  * NVT by velocity rescaling to the state's temperature every
    ``--every`` steps (the paper names no thermostat);
  * every ``--every`` steps a sample of E/N = (E2 + E2_tail + E3) / N and
    P = (2 K + W2 + W3) / (3 V) + P2_tail (long-range corrections on the pair
    terms only) and of the pair-distance histogram (r < 2.5, the cell edge).

    python -m paper_2510_21230_gb300.replay --melt 25000 --prod 25000

prints one JSON line per (state, run) with the averages, their standard
errors (block averages), the first RDF peak and the paper's value of the
same entry of Table 1phase for context.
"""
import argparse
import json
import math
import os
import sys
import time

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2510_21230_gb300 import analysis, atm3, build, synth  # noqa: E402

BOX, RC, DT = 12.5, 2.5, 0.004
NU_PAPER = 0.072
STATES = [dict(name="T1.033_rho0.65", T=1.033, rho=0.65, n=1270),
          dict(name="T0.746_rho0.817", T=0.746, rho=0.817, n=1596)]

# Table 1phase (E/N, P) for context: per state, per run
TABLE_1PHASE = {
    "T1.033_rho0.65": {("3c01", "pair"): (-4.37965, 0.10406), ("3c01", "product"): (-4.37695, 0.10933),
                       ("3c18", "pair"): (-4.38009, 0.10682), ("3c18", "product"): (-4.37872, 0.11725),
                       ("3c08", "pair"): (-4.38044, 0.10891), ("3c08", "product"): (-4.37934, 0.10601),
                       ("lj", None): (-4.5395, -0.1140)},
    "T0.746_rho0.817": {("3c01", "pair"): (-5.62938, 0.48192), ("3c01", "product"): (-5.62655, 0.48764),
                        ("3c18", "pair"): (-5.63040, 0.47474), ("3c18", "product"): (-5.62686, 0.48936),
                        ("3c08", "pair"): (-5.63252, 0.47269), ("3c08", "product"): (-5.63139, 0.47222),
                        ("lj", None): (-5.8932, -0.09705)},
}


def _block_error(x, nblocks=10):
    x = np.asarray(x, dtype=np.float64)
    if x.size < 2 * nblocks:
        return float("nan")
    m = x[: x.size // nblocks * nblocks].reshape(nblocks, -1).mean(axis=1)
    return float(m.std(ddof=1) / math.sqrt(nblocks))


def _run(sys_, nsteps, every, trav, trunc, prec, temps, tails, sample, rdf_bins):
    """nsteps in chunks of ``every``; thermostat after each chunk; samples."""
    V = BOX ** 3
    E = [[] for _ in STATES]
    P = [[] for _ in STATES]
    if sample:
        sys_.rdf_reset()
    for _ in range(max(1, nsteps // every)):
        sys_.step(every, trav, trunc, prec)
        if sample:
            for r, res in enumerate(sys_.results()):
                n = STATES[r]["n"]
                E[r].append((res["e2"] + tails[r][0] + res["e3"]) / n)
                P[r].append((2.0 * res["ekin"] + res["w2"] + res["w3"]) / (3.0 * V) + tails[r][1])
            sys_.rdf_accumulate(RC, rdf_bins)
        sys_.thermostat(temps)
    return E, P


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--melt", type=int, default=25000)
    p.add_argument("--prod", type=int, default=25000)
    p.add_argument("--every", type=int, default=10)
    p.add_argument("--runs", default="3c01:pair,3c01:product,3c18:pair,3c18:product,3c08:pair,3c08:product")
    p.add_argument("--prec", default="fp64", choices=["fp64", "fp32c"])
    p.add_argument("--rdf-bins", type=int, default=250)
    p.add_argument("--seed", type=int, default=51)
    p.add_argument("--out", default=None, help="write the RDFs (npz) here")
    a = p.parse_args()
    build.build()
    rng = np.random.default_rng(a.seed)
    xs, vs = [], []
    for st in STATES:
        xs.append(synth.simple_cubic_positions(st["n"], BOX, rng))
        vs.append(synth.maxwell_boltzmann(st["n"], st["T"], rng))
    x = np.ascontiguousarray(np.concatenate(xs, axis=1))
    v = np.ascontiguousarray(np.concatenate(vs, axis=1))
    ns = [st["n"] for st in STATES]
    temps = [st["T"] for st in STATES]
    tails = [atm3.lj_tail(BOX, st["n"], rc=RC) for st in STATES]
    rdfs = {}
    t0 = time.perf_counter()

    def report(tag, key, E, P, sys_):
        counts, samples = sys_.rdf_get(a.rdf_bins)
        for r, st in enumerate(STATES):
            rr, g = analysis.rdf(counts[r], samples, st["n"], BOX ** 3, RC)
            rdfs["%s/%s" % (st["name"], tag)] = g
            k = int(np.argmax(g))
            ref = TABLE_1PHASE[st["name"]].get(key)
            print(json.dumps({"state": st["name"], "run": tag, "steps": a.prod, "every": a.every,
                              "E_per_N": float(np.mean(E[r])), "E_err": _block_error(E[r]),
                              "P": float(np.mean(P[r])), "P_err": _block_error(P[r]),
                              "rdf_peak": [float(rr[k]), float(g[k])],
                              "paper_table_1phase": ref,
                              "elapsed_s": round(time.perf_counter() - t0, 1)}), flush=True)

    # melting and the nu = 0 reference (LJ only; the ATM kernels contribute 0)
    with atm3.AtmSystem(BOX, ns, rc=RC, nu=0.0, dt=DT) as s:
        s.set_state(x, v)
        s.set_options(graph=True)
        _run(s, a.melt, a.every, "3c08", "pair", "fp32c", temps, tails, False, a.rdf_bins)
        E, P = _run(s, a.prod, a.every, "3c08", "pair", "fp32c", temps, tails, True, a.rdf_bins)
        report("lj_nu0", ("lj", None), E, P, s)
        x, v = s.get_state()
    for item in a.runs.split(","):
        trav, trunc = item.split(":")
        with atm3.AtmSystem(BOX, ns, rc=RC, nu=NU_PAPER, dt=DT) as s:
            s.set_state(x, v)
            s.set_options(graph=True)
            E, P = _run(s, a.prod, a.every, trav, trunc, a.prec, temps, tails, True, a.rdf_bins)
            report("%s_%s" % (trav, trunc), (trav, trunc), E, P, s)
    if a.out:
        np.savez(a.out, r=analysis.rdf(np.zeros(a.rdf_bins), 1, 1, 1.0, RC)[0], **rdfs)


if __name__ == "__main__":
    main()
