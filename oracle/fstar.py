"""f* of the benchmark scenes, for the 1 % cost tolerance of bench.py.

The paper's performance profiles (appendix) measure the time to reach
f_tau = f* + tau (f0 - f*), f* the best cost any solver reaches.  The FP64
oracle run to convergence stands for that solver here: Levenberg-Marquardt to
at most 50 iterations with a tight CG forcing tolerance (eta = 1e-3) and
function tolerance 1e-6 (Sec. 6.1 settings otherwise).  Both arms of bench.py
take f* from the table this prints, so that they time the same target.

    python oracle/fstar.py medium:0 large:0      # prints the table entries
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def fstar(config, seed, threads=None):
    import oracle
    from paper_2103_01843_gb300.synth import make_scene
    oracle.set_threads(threads or oracle.max_threads())
    s = make_scene(config, seed)
    t0 = time.perf_counter()
    _, _, log = oracle.lm(s, max_iters=50, dense=False, cg_eta=1e-3, func_tol=1e-6)
    best = min([e["new_cost"] for e in log if e["accepted"]] + [log[0]["cost"]])
    return best, log[0]["cost"], len(log), time.perf_counter() - t0


def main(argv):
    for item in argv or ["medium:0"]:
        config, seed = item.split(":")
        f, f0, n, dt = fstar(config, int(seed))
        print(f'    ("{config}", {int(seed)}): {f!r},  # f0 {f0:.9g}, {n} LM iterations, {dt:.0f} s', flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
