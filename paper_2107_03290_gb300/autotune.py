"""Autotuner of the batched sort (ls_sort_batch), run on a GB300.

Arrays of more than 8192 keys are first split by a line through their own key
range; the number of keys per sub-bucket that split aims at decides which
in-bucket class finishes them and how many further splits follow.  For each
array-size class (at most 65,536 keys, at most 524,288, larger) this sweeps
that target on the arrays of the batched workload that fall in the class (4096
float64 arrays, lognormal sizes with median 64K clipped to [1K, 4M], each
N(0,1), U[0,1) or Zipf(1.1) over 10^4 values), times ls_sort_batch_ex with CUDA
events (inputs restored from a device copy outside the timing, median of
several runs), checks the fastest setting's output, and writes the table
csrc/ls_tuned.h that the library compiles in.  For comparison it also times
the learned alternative on the same arrays (a sampled RMI per array: ls_sort
on each in turn) and records it in the table's comment.

  python -m paper_2107_03290_gb300.autotune [--out PATH] [--reps 5]
"""
from __future__ import annotations

import argparse
import datetime
import os
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(_HERE))

CLASS_MAX = [65536, 524288, 0xFFFFFFFF]
CANDIDATES = [512, 768, 1024, 1536, 2048, 2560, 3072, 4096]


def _class_of(m: int) -> int:
    c = 0
    while c < 2 and m > CLASS_MAX[c]:
        c += 1
    return c


def sweep(reps: int = 5, count: int = 4096):
    import torch

    import lsgen
    import paper_2107_03290_gb300 as ls
    ls.build()
    ls.load()
    arrays = lsgen.batch_arrays(count, seed=6)
    st = torch.cuda.current_stream()
    result = {}
    for c in range(3):
        sel = [a for a in arrays if a.size > 8192 and _class_of(a.size) == c]
        if not sel:
            continue
        offs = np.concatenate([[0], np.cumsum([a.size for a in sel])]).astype(np.int64)
        pristine = torch.from_numpy(np.concatenate(sel)).cuda()
        work = torch.empty_like(pristine)
        views = [work[offs[i]:offs[i + 1]] for i in range(len(sel))]
        times = {}
        for tgt in CANDIDATES:
            split = [0, 0, 0]
            split[c] = tgt
            ms = []
            for r in range(reps + 1):
                work.copy_(pristine)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                ls.sort_batch_(views, split_target=split)
                e1.record(st)
                e1.synchronize()
                if r:
                    ms.append(e0.elapsed_time(e1))
            times[tgt] = float(np.median(ms))
        best = min(times, key=times.get)
        # the learned alternative: a sampled RMI per array (ls_sort on each array
        # in turn, same stream), timed once after a warm-up pass
        learned = []
        for r in range(2):
            work.copy_(pristine)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for v in views:
                ls.sort_(v)
            e1.record(st)
            e1.synchronize()
            learned.append(e0.elapsed_time(e1))
        # the chosen setting must sort every array of the class
        split = [0, 0, 0]
        split[c] = best
        work.copy_(pristine)
        ls.sort_batch_(views, split_target=split)
        torch.cuda.synchronize()
        out = work.cpu().numpy()
        for i, a in enumerate(sel):
            if not np.array_equal(out[offs[i]:offs[i + 1]], np.sort(a)):
                raise RuntimeError(f"class {c}: array {i} not sorted with target {best}")
        result[c] = {"arrays": len(sel), "keys": int(offs[-1]), "ms": times, "best": best,
                     "learned_ms": float(learned[-1])}
        del pristine, work, views
        torch.cuda.empty_cache()
    return result


def write_header(result: dict, path: str, gpu: str):
    best = [result.get(c, {}).get("best", 3072) for c in range(3)]
    lines = [
        "// Tuned parameters of the batched sort, per array-size class: the keys per",
        "// sub-bucket aimed at by the first range split of an array.  Written by",
        "// paper_2107_03290_gb300/autotune.py (the sweep and the GPU it ran on are in",
        "// the comment below); edit by re-running it, not by hand.",
        "//",
        f"// {gpu}, {datetime.date.today().isoformat()}: ls_sort_batch_ex on the batched",
        "// workload's arrays of each class, median ms per call:",
    ]
    for c in range(3):
        r = result.get(c)
        if not r:
            continue
        row = ", ".join(f"{t}: {v:.3f}" for t, v in r["ms"].items())
        lines.append(f"//   class {c} ({r['arrays']} arrays, {r['keys']} keys): {row}")
        lines.append(f"//     (a sampled RMI per array instead, ls_sort on each: {r['learned_ms']:.1f} ms)")
    lines += [
        "#pragma once",
        "#include <stdint.h>",
        "",
        "namespace ls {",
        "constexpr uint32_t TUNED_CLASS_MAX[3] = {65536u, 524288u, 0xFFFFFFFFu};  // largest array per class",
        f"constexpr uint32_t TUNED_SPLIT_TARGET[3] = {{{best[0]}u, {best[1]}u, {best[2]}u}};",
        "}  // namespace ls",
        "",
    ]
    with open(path, "w") as f:
        f.write("\n".join(lines))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(_HERE, "csrc", "ls_tuned.h"))
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    import torch
    res = sweep(args.reps)
    write_header(res, args.out, torch.cuda.get_device_name(0))
    for c, r in sorted(res.items()):
        print(f"class {c}: best {r['best']}  " + "  ".join(f"{t}:{v:.3f}" for t, v in r["ms"].items())
              + f"  learned per array: {r['learned_ms']:.1f}")


if __name__ == "__main__":
    main()
