"""Basin hopping over the S-box circuits: CGP drift, then windowed resynthesis.

Each step takes the current circuit of one S-box, lets cgpopt drift across
circuits of (about) the same size for a minute, allowing a few extra gates
now and then, and hands the circuit it drifted to to ``sboxgen --polish``,
which rebuilds fanout-free cones with fewer gates.  Whatever comes out at no
more than one gate above the best becomes the next start point (most of the
time), so the walk leaves the local optimum the searches stop in.  Every
strictly smaller circuit is kept.

    python hop_search.py --start sbox_circuits.json --workers 8 --minutes 60 --out best_dir

Builds cgpopt and sboxgen with gcc into the output directory, writes
``best_s<k>.json`` for every S-box that improved, and prints each
improvement.  merge_circuits.py then folds the results into
sbox_circuits.json.
"""
import argparse
import concurrent.futures as cf
import json
import os
import random
import subprocess
import time

HERE = os.path.dirname(os.path.abspath(__file__))


def build(out_dir):
    tools = {}
    for name in ("cgpopt", "sboxgen"):
        exe = os.path.join(out_dir, name)
        subprocess.run(["gcc", "-O2", "-o", exe, os.path.join(HERE, name + ".c")], check=True)
        tools[name] = exe
    return tools


def step(tools, work, box, circuit, seed):
    start = os.path.join(work, "start_s%d_%d.json" % (box, seed))
    drift = os.path.join(work, "drift_s%d_%d.json" % (box, seed))
    best = os.path.join(work, "cgp_s%d_%d.json" % (box, seed))
    pol = os.path.join(work, "pol_s%d_%d.json" % (box, seed))
    with open(start, "w") as f:
        json.dump([circuit], f)
    rng = random.Random(seed)
    subprocess.run([tools["cgpopt"], start, str(box), str(seed), "60", str(rng.choice([6, 10, 14])), best,
                    str(rng.choice([1, 2, 3])), drift], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    subprocess.run([tools["sboxgen"], "--polish", drift if os.path.exists(drift) else start, str(box), str(seed),
                    "90", pol], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    found = []
    for path in (best, drift, pol):
        if os.path.exists(path):
            try:
                with open(path) as f:
                    found += [c for c in json.load(f) if c["sbox"] == box]
            except ValueError:
                pass
    for path in (start, best, drift, pol):
        if os.path.exists(path):
            os.remove(path)
    return found


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--start", default=os.path.join(HERE, "sbox_circuits.json"))
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 4)
    ap.add_argument("--minutes", type=float, default=60.0)
    ap.add_argument("--out", default="hop_out")
    ap.add_argument("--seed", type=int, default=1)
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    work = os.path.join(args.out, "work")
    os.makedirs(work, exist_ok=True)
    tools = build(args.out)
    rng = random.Random(args.seed)
    with open(args.start) as f:
        best = {c["sbox"]: c for c in json.load(f)}
    cur = dict(best)
    deadline = time.time() + 60 * args.minutes
    it = 0
    with cf.ThreadPoolExecutor(args.workers) as ex:
        running = {}
        while running or time.time() < deadline:
            while time.time() < deadline and len(running) < args.workers:
                box = 1 + it % 8
                it += 1
                running[ex.submit(step, tools, work, box, cur[box], rng.randrange(1 << 30))] = box
            done, _ = cf.wait(list(running), return_when=cf.FIRST_COMPLETED)
            for fut in done:
                box = running.pop(fut)
                for c in fut.result():
                    if len(c["gates"]) < len(best[box]["gates"]):
                        best[box] = c
                        with open(os.path.join(args.out, "best_s%d.json" % box), "w") as f:
                            json.dump([c], f)
                        print(time.strftime("%H:%M:%S"), "S%d: %d gates" % (box, len(c["gates"])), flush=True)
                    if len(c["gates"]) <= len(best[box]["gates"]) + 1 and rng.random() < 0.7:
                        cur[box] = c
                    elif rng.random() < 0.3:
                        cur[box] = best[box]


if __name__ == "__main__":
    main()
