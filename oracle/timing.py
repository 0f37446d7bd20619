"""Host timing of the FP64 oracle (test infrastructure, as it stands): seconds
per RK2 step of the 256^3-style Taylor-Green run (nu = 1/1600, dt = 2e-3) at
the sizes and OpenMP thread counts given, single-threaded and loop-parallel
(the oracle's OpenMP loops over independent lines and modes).  One untimed
step first, then the timed steps; one JSON line per case.

    python -m oracle.timing 64:1:5 64:all:5 256:all:2     # N:threads:steps
"""
import json
import os
import sys
import time

import oracle


def main(argv):
    from paper_1003_4322_gb300 import inputs
    for spec in argv:
        n_s, th_s, steps_s = spec.split(":")
        n, steps = int(n_s), int(steps_s)
        want = (os.cpu_count() or 1) if th_s == "all" else int(th_s)
        threads = oracle.set_threads(want)
        p = oracle.Params(n=n, nu=1 / 1600, dt=2e-3)
        a = oracle.step(inputs.taylor_green_state(n), p, 1)
        t0 = time.perf_counter()
        oracle.step(a, p, steps)
        s = (time.perf_counter() - t0) / steps
        print(json.dumps({"n": n, "threads": threads, "steps": steps, "s_per_step": s,
                          "steps_per_s": 1 / s, "host_cpus": os.cpu_count()}), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["32:1:10", "32:all:10", "64:1:3", "64:all:5", "128:1:1", "128:all:3",
                          "256:all:2"])
