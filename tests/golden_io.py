"""Reader for the hand-worked fixtures under tests/golden/."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_worked_example(name: str = "worked_example.txt"):
    """Returns (windows, nonzeros, stats_after): windows is a list of
    (src, dst) uint32 arrays, nonzeros is (keys, counts) uint64, and
    stats_after maps window index -> 9-tuple."""
    windows, cur, nz, stats = [], [], [], {}
    mode = None
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] in ("packets", "nonzeros"):
                mode = tok[0]
                continue
            if tok[0] == "window":
                windows.append(cur)
                cur = []
                continue
            if tok[0] == "end":
                if mode == "packets":
                    windows.append(cur)
                    cur = []
                mode = None
                continue
            if tok[0] == "stats_after_window":
                stats[int(tok[1])] = tuple(int(x) for x in tok[2:])
                continue
            if mode == "packets":
                cur.append((int(tok[0]), int(tok[1])))
            elif mode == "nonzeros":
                nz.append(((int(tok[0]) << 32) | int(tok[1]), int(tok[2])))
    wins = [(np.array([p[0] for p in w], np.uint32), np.array([p[1] for p in w], np.uint32))
            for w in windows]
    keys = np.array([k for k, _ in nz], np.uint64)
    counts = np.array([c for _, c in nz], np.uint64)
    return wins, (keys, counts), stats


def read_anonymize_example(name: str = "anonymize_example.txt"):
    """Returns (src, dst, rnd, out_src, out_dst) of the hand-worked
    anonymization fixture."""
    sec, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] in ("packets", "random", "anonymized"):
                cur = tok[0]
                sec[cur] = []
                continue
            if tok[0] == "end":
                cur = None
                continue
            sec[cur].append([int(x) for x in tok])
    p = np.array(sec["packets"], dtype=np.uint64)
    a = np.array(sec["anonymized"], dtype=np.uint64)
    r = np.array([x[0] for x in sec["random"]], dtype=np.uint64)
    return (p[:, 0].astype(np.uint32), p[:, 1].astype(np.uint32), r,
            a[:, 0].astype(np.uint32), a[:, 1].astype(np.uint32))
