"""Write tests/golden/condensation_stats.json: droplet statistics of the FP64 oracle on
the 128 x 32 cut-down channels (the condensation measure of the Section 3.3 channel).

Calls only the oracle (oracle/ and oracle/droplets.py) and the seeded input
generator.  Two workloads, each from its seeded initial density:
  channel_128x32 : walls at 0.80 Tc, 50000 updates, statistics every 10000;
  cold_128x32    : walls at 0.65 Tc, statistics at 5000, 10000 and 15000 updates.
Liquid threshold: the mean of the coexistence densities at 0.86 Tc; condensed mass
relative to the vapour density rho_v(0.86 Tc).

    python tests/golden/make_condensation_stats.py
"""
import json
import os
import sys
from multiprocessing import get_context

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

PLAN = {"channel_128x32": [10000, 20000, 30000, 40000, 50000],
        "cold_128x32": [5000, 10000, 15000]}


def run(name):
    import oracle
    from oracle.droplets import droplet_stats
    from paper_1803_01756_gb300 import inputs
    w = inputs.workload(name)
    o = oracle.Oracle(w["nx"], w["ny"], w["params"])
    o.set_fields(inputs.initial_density(w))
    thr = 0.5 * (inputs.RHO_L_086 + inputs.RHO_V_086)
    out = {}
    for t in PLAN[name]:
        o.step(t - o.t)
        rho = o.fields()[0]
        st = droplet_stats(rho, thr, inputs.RHO_V_086)
        st["status"] = int(o.status)
        st["rho_max"] = float(rho.max())
        out[str(t)] = st
    return name, out


def main():
    with get_context("spawn").Pool(len(PLAN)) as pool:
        res = dict(pool.map(run, sorted(PLAN)))
    res["_about"] = ("FP64 oracle droplet statistics on 128 x 32 cut-downs; written by "
                     "tests/golden/make_condensation_stats.py")
    with open(os.path.join(HERE, "condensation_stats.json"), "w") as fh:
        json.dump(res, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
