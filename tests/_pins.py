"""A battery of checks that pins an oracle build to things other than itself.

``run_battery(orc)`` returns a list of failure strings (empty = every pin holds).  The
same battery runs on the real oracle (must pass) and on planted mutants of its C source
(each must fail), which shows that the pins can see a plausible mistake.
"""
from __future__ import annotations

import itertools

import numpy as np

import synth
from _defs import check_invariants, closed_forms, load_golden, scipy_labels


def _all_images(h, w):
    n = h * w
    for bits in range(1 << n):
        yield np.array([(bits >> i) & 1 for i in range(n)], dtype=np.uint8).reshape(h, w)


def _variants(orc):
    """(name, conn, fn) for every oracle entry point."""
    return [
        ("cclremsp8", 8, lambda im: orc.cclremsp(im, 8)),
        ("cclremsp4", 4, lambda im: orc.cclremsp(im, 4)),
        ("aremsp", 8, lambda im: orc.aremsp(im)),
        ("paremsp1", 8, lambda im: orc.paremsp(im, 1)),
        ("paremsp3", 8, lambda im: orc.paremsp(im, 3)),
        ("paremsp8", 8, lambda im: orc.paremsp(im, 8)),
        ("bfs8", 8, lambda im: orc.bfs(im, 8)),
        ("bfs4", 4, lambda im: orc.bfs(im, 4)),
    ]


def run_battery(orc, exhaustive=((3, 3), (2, 6), (4, 4)), stop_early=False):
    errs = []

    def fail(msg):
        errs.append(msg)
        return stop_early

    variants = _variants(orc)
    # 1. hand-derived fixtures
    for g in load_golden():
        for name, conn, fn in variants:
            lab, k = fn(g["image"])
            exp, ek = (g["labels8"], g["k8"]) if conn == 8 else (g["labels4"], g["k4"])
            if k != ek or not np.array_equal(lab, exp):
                if fail(f"golden {g['name']} {name}: K={k} expected {ek}"):
                    return errs
    # 2. closed forms
    for cname, img, conn, ek, exp in closed_forms():
        for name, vconn, fn in variants:
            if vconn != conn:
                continue
            lab, k = fn(img)
            if k != ek or (exp is not None and not np.array_equal(lab, exp)):
                if fail(f"closed form {cname} {name}: K={k} expected {ek}"):
                    return errs
    # 3. exhaustive tiny images against scipy (library flood fill)
    for (h, w) in exhaustive:
        for img in _all_images(h, w):
            ref = {8: scipy_labels(img, 8), 4: scipy_labels(img, 4)}
            for name, conn, fn in variants:
                lab, k = fn(img)
                if k != ref[conn][1] or not np.array_equal(lab, ref[conn][0]):
                    if fail(f"exhaustive {h}x{w} {name} on {img.ravel().tolist()}"):
                        return errs
                    break
    # 4. random images, padded pitch (padding bytes are non-zero), odd shapes
    shapes = [(1, 37), (37, 1), (2, 2), (7, 13), (31, 64), (65, 33), (128, 129), (257, 96)]
    for (h, w), p, seed in itertools.product(shapes, (0.1, 0.45, 0.6, 0.9), (11,)):
        img = synth.bernoulli(h, w, p, seed + h * 1000 + w)
        padded = synth.pad_pitch(img, w + 5 + (h % 3))[:, :w]
        for conn in (8, 4):
            ref_lab, ref_k = scipy_labels(img, conn)
            for name, vconn, fn in variants:
                if vconn != conn:
                    continue
                for src in (img, padded):
                    lab, k = fn(src)
                    if k != ref_k or not np.array_equal(lab, ref_lab):
                        if fail(f"random {h}x{w} p={p} {name}: K={k} expected {ref_k}"):
                            return errs
                        break
                    inv = check_invariants(img, lab, k, conn)
                    if inv:
                        if fail(f"random {h}x{w} p={p} {name}: {inv}"):
                            return errs
                        break
    return errs
