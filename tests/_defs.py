"""Definition-level checks shared by the tests.

Everything here is written from the problem statement (Section III of the paper): object
pixels (non-zero bytes) that are 4- or 8-adjacent belong to one component; the numbering
used throughout is background 0 and components 1..K in raster order of first pixels.
Nothing here calls the oracle or the GPU library.
"""
from __future__ import annotations

import os
from collections import deque

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

N8 = [(-1, -1), (-1, 0), (-1, 1), (0, -1), (0, 1), (1, -1), (1, 0), (1, 1)]
N4 = [(-1, 0), (0, -1), (0, 1), (1, 0)]


def bfs_py(img: np.ndarray, conn: int = 8):
    """Brute-force flood fill in pure Python (tiny images only)."""
    h, w = img.shape
    nb = N8 if conn == 8 else N4
    lab = np.zeros((h, w), dtype=np.int32)
    k = 0
    for y in range(h):
        for x in range(w):
            if img[y, x] == 0 or lab[y, x]:
                continue
            k += 1
            lab[y, x] = k
            q = deque([(y, x)])
            while q:
                cy, cx = q.popleft()
                for dy, dx in nb:
                    ny, nx = cy + dy, cx + dx
                    if 0 <= ny < h and 0 <= nx < w and img[ny, nx] and not lab[ny, nx]:
                        lab[ny, nx] = k
                        q.append((ny, nx))
    return lab, k


def first_occurrence(labels: np.ndarray):
    """Renumber arbitrary positive labels 1..K by first raster occurrence (numpy)."""
    flat = np.ascontiguousarray(labels).ravel()
    out = np.zeros(flat.shape, dtype=np.int32)
    m = flat > 0
    if not m.any():
        return out.reshape(labels.shape), 0
    uniq, first = np.unique(flat[m], return_index=True)
    order = np.argsort(first, kind="stable")
    mapping = np.zeros(int(flat.max()) + 1, dtype=np.int32)
    mapping[uniq[order]] = np.arange(1, uniq.size + 1, dtype=np.int32)
    out = mapping[flat]
    return out.reshape(labels.shape), int(uniq.size)


def scipy_labels(img: np.ndarray, conn: int = 8):
    """scipy.ndimage.label with the 3x3 (8) or cross (4) structure, renumbered."""
    import scipy.ndimage as ndi

    st = np.ones((3, 3), dtype=bool) if conn == 8 else ndi.generate_binary_structure(2, 1)
    lab, n = ndi.label(np.asarray(img) != 0, structure=st)
    out, k = first_occurrence(lab)
    assert k == n
    return out, k


def check_invariants(img: np.ndarray, labels: np.ndarray, k: int, conn: int = 8):
    """Checks that hold for any correct answer at any size.  Returns failure strings."""
    errs = []
    fgm = np.asarray(img) != 0
    lab = np.asarray(labels)
    if lab.shape != fgm.shape:
        return [f"shape {lab.shape} != {fgm.shape}"]
    if (lab[~fgm] != 0).any():
        errs.append("background pixel with non-zero label")
    if (lab[fgm] <= 0).any():
        errs.append("object pixel with label <= 0")
    offs = [(0, 1), (1, -1), (1, 0), (1, 1)] if conn == 8 else [(0, 1), (1, 0)]
    h, w = fgm.shape
    for dy, dx in offs:
        y0, y1 = 0, h - dy
        xa0, xa1 = max(0, -dx), w - max(0, dx)
        a = (slice(y0, y1), slice(xa0, xa1))
        b = (slice(y0 + dy, y1 + dy), slice(xa0 + dx, xa1 + dx))
        both = fgm[a] & fgm[b]
        if (lab[a][both] != lab[b][both]).any():
            errs.append(f"adjacent object pixels ({dy},{dx}) with different labels")
    vals = lab[fgm]
    if vals.size:
        uniq, first = np.unique(vals, return_index=True)
        if uniq.size != k or uniq[0] != 1 or uniq[-1] != k:
            errs.append(f"labels are not exactly 1..K (K={k}, distinct={uniq.size})")
        elif (np.diff(first) <= 0).any():
            errs.append("first occurrences not in raster order")
    elif k != 0:
        errs.append(f"no object pixels but K={k}")
    return errs


def load_golden():
    """Parse tests/golden/*.txt into dicts: name, image, labels8, k8, labels4, k4."""
    out = []
    for fn in sorted(os.listdir(GOLDEN_DIR)):
        if not fn.endswith(".txt"):
            continue
        sections, cur = {}, None
        with open(os.path.join(GOLDEN_DIR, fn)) as f:
            for line in f:
                line = line.strip()
                if not line or line.startswith("#"):
                    continue
                parts = line.split()
                if parts[0] in ("image", "labels8", "labels4"):
                    cur = parts[0]
                    sections[cur] = {"k": int(parts[1]) if len(parts) > 1 else None, "rows": []}
                else:
                    sections[cur]["rows"].append([int(v) for v in parts])
        img = np.array(sections["image"]["rows"], dtype=np.uint8)
        rec = {"name": fn[:-4], "image": img}
        for key in ("labels8", "labels4"):
            rec[key] = np.array(sections[key]["rows"], dtype=np.int32)
            rec["k" + key[-1]] = sections[key]["k"]
        out.append(rec)
    return out


def closed_forms():
    """(name, image, conn, expected K, optional expected labels) with known answers."""
    import synth

    cases = []
    for h, w in [(1, 1), (1, 7), (7, 1), (5, 5), (6, 9), (33, 65), (64, 257)]:
        cases.append((f"zeros_{h}x{w}", np.zeros((h, w), np.uint8), 8, 0, np.zeros((h, w), np.int32)))
        cases.append((f"ones_{h}x{w}", np.ones((h, w), np.uint8), 8, 1, np.ones((h, w), np.int32)))
        cases.append((f"ones4_{h}x{w}", np.ones((h, w), np.uint8), 4, 1, np.ones((h, w), np.int32)))
        cb = synth.checkerboard(h, w)
        if h >= 2 and w >= 2:
            cases.append((f"checker_{h}x{w}", cb, 8, 1, cb.astype(np.int32)))
        # dot lattice: label(2i, 2j) = i*ceil(W/2) + j + 1
        dl = synth.dot_lattice(h, w)
        exp = np.zeros((h, w), np.int32)
        cw = (w + 1) // 2
        for i in range((h + 1) // 2):
            for j in range(cw):
                exp[2 * i, 2 * j] = i * cw + j + 1
        cases.append((f"dots_{h}x{w}", dl, 8, ((h + 1) // 2) * cw, exp))
        cases.append((f"dots4_{h}x{w}", dl, 4, ((h + 1) // 2) * cw, exp))
        # 4-connectivity: a checkerboard's object pixels touch only diagonally, so each is
        # its own component, numbered in raster order
        exp = np.zeros((h, w), np.int32)
        exp[cb != 0] = np.arange(1, int((cb != 0).sum()) + 1)
        cases.append((f"checker4_{h}x{w}", cb, 4, int((cb != 0).sum()), exp))
        # the main diagonal: one component under 8-connectivity, min(h, w) under 4
        dg = np.eye(h, w, dtype=np.uint8)
        n = min(h, w)
        cases.append((f"diag_{h}x{w}", dg, 8, 1, dg.astype(np.int32)))
        exp = np.zeros((h, w), np.int32)
        exp[np.arange(n), np.arange(n)] = np.arange(1, n + 1)
        cases.append((f"diag4_{h}x{w}", dg, 4, n, exp))
        sr = synth.striped_rows(h, w)
        exp = np.zeros((h, w), np.int32)
        exp[0::2, :] = (np.arange(0, h, 2) // 2 + 1)[:, None]
        cases.append((f"rows_{h}x{w}", sr, 8, (h + 1) // 2, exp))
        cases.append((f"rows4_{h}x{w}", sr, 4, (h + 1) // 2, exp))
        sp = synth.serpentine(h, w)
        if w >= 2:
            cases.append((f"serpentine_{h}x{w}", sp, 8, 1, sp.astype(np.int32)))
            cases.append((f"serpentine4_{h}x{w}", sp, 4, 1, sp.astype(np.int32)))
    for w in (1, 2, 5, 8, 31):
        cb = synth.checkerboard(1, w)
        exp = np.zeros((1, w), np.int32)
        exp[0, 0::2] = np.arange(1, (w + 1) // 2 + 1)
        cases.append((f"checker_1x{w}", cb, 8, (w + 1) // 2, exp))
    return cases
