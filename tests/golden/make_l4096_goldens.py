"""Write the stored trajectory records of the L = 4096, 10^4-sweep workloads.

Calls only the CPU oracle (``oracle/``): the flat start (Sec. 2.1 of
arXiv:1204.5072), the decomposed schedule (Sec. 3 dead-border tiles of
128 x 128 sites with a random origin per sweep, Sec. 3.1 single-hit rounds),
seed 1, sample 0, run with the tiles of each sweep spread over the host's
cores (the same result as the single-threaded sweep). At every sampling time
t of the run (64 log-spaced times, t_k = ceil(10^(k log10(T)/63)), plus t = 0)
it records

    t  S1  S2  h00  sha256(packed slopes)

S1 and S2 are the exact sums of h and h^2 over the L^2 sites in the gauge
h(0,0) = 0 (eq. Wdef), h00 the absolute height of site (0,0), and the digest
is taken over the canonical packed slope words (row j in L/16 little-endian
uint32 words, sigma_x of site i at bit 2(i%16), sigma_y at bit 2(i%16)+1).

Usage:  python tests/golden/make_l4096_goldens.py P Q OUT [--threads N]
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O          # noqa: E402
from synth import inputs as I           # noqa: E402

L, TILE, SEED, SAMPLE, MCS = 4096, 128, 1, 0, 10_000


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("p", type=float)
    ap.add_argument("q", type=float)
    ap.add_argument("out")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--mcs", type=int, default=MCS)
    a = ap.parse_args()
    st = O.State.flat(L)
    lines = [f"# octahedron KPZ, L={L}, p={a.p}, q={a.q}, flat start, seed {SEED}, sample {SAMPLE}, "
             f"tiles {TILE}x{TILE}, {a.mcs} sweeps",
             "# written by tests/golden/make_l4096_goldens.py from the CPU oracle alone",
             "# t S1 S2 h00 sha256(packed slopes)"]
    t0 = time.time()
    for t in I.sample_times(a.mcs):
        if t > st.t:
            st.run_threads(t - st.t, TILE, TILE, a.p, a.q, SEED, SAMPLE, threads=a.threads)
        s1, s2 = st.sums()
        digest = hashlib.sha256(st.packed().tobytes()).hexdigest()
        lines.append(f"{t} {s1} {s2} {st.h00} {digest}")
        print(f"t={t} S1={s1} S2={s2} h00={st.h00} ({time.time() - t0:.0f} s)", flush=True)
    tmp = a.out + ".tmp"
    with open(tmp, "w") as f:
        f.write("\n".join(lines) + "\n")
    os.replace(tmp, a.out)


if __name__ == "__main__":
    main()
