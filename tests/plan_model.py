"""A data-parallel formulation of the host planner, for batches planned
without sharing and without bit slicing (HEDL_NO_CSE | HEDL_NO_SLICE, fillers
not staged) — TEST INFRASTRUCTURE.

Every step is either independent per hypothesis or a prefix sum, a stable
sort or a reduction over hypotheses or segments, which is the shape that a
device-side planner (one thread per hypothesis, then scans) takes:

1. per hypothesis, in instruction order: the expression tree (without
   sharing, one node per instruction), which role fillers are materialised
   (every filler that is not a concept, plus the operand with the larger
   stack need wherever an AND / OR would need more than 15 stack entries),
   the stack need of every node;
2. per hypothesis: one segment per materialised node and one for the root,
   each emitted in post-order with the larger-need operand first; the slots
   it reads, its first role restriction's key, its staged filler, its level
   (one above the slots it reads), its algorithmic bytes;
3. prefix sums: global slot ids (materialised nodes in instruction order),
   segment ids (all materialised segments, then the roots), code offsets,
   dependency offsets;
4. a reduction (segments per level that walk a role) chooses the tile
   shape; a stable sort by (level, role key) orders the work queue.

The image it writes is compared byte for byte with the library's
(`hedl_plan_image`), so the formulation is pinned before a GPU kernel
implements it.  It reads the library's layout constants from its header
declarations; it evaluates nothing.
"""
from __future__ import annotations

import struct
from typing import List, Sequence

import numpy as np

from synth import programs as P

# instruction kinds of a segment (the interpreter's D_* codes) and references
D_ATOM, D_TOP, D_BOT, D_NOT, D_AND, D_OR, D_ROLE, D_DATA, D_SLOT = 1, 2, 3, 4, 5, 6, 7, 12, 32
REF_SLOT, REF_NEG = 0x80000000, 0x40000000
NO_SLOT = NO_HYP = NO_FILLER = 0xFFFFFFFF
STACK_MAX = 16
HEADER = "<12I11Q"            # PlanHeader: 12 uint32 counts, 11 uint64 offsets / timeout
SEG = "<8I"                   # code_off, code_len, out_slot, hyp, dep_off, dep_cnt, filler, kind
GROUP = "<4I"                 # item_begin, seg_begin, n_segs, level
INSN = "<4I"                  # op, a, b, ref


def _arity(op: int) -> int:
    if op in (P.NOT,) + P.ROLE_OPS:
        return 1
    if op in (P.AND, P.OR):
        return 2
    return 0


class Hyp:
    """Steps 1-2 for one program (local node, slot and segment numbering)."""

    def __init__(self, prog: Sequence[int], kb):
        self.nodes = []
        st: List[int] = []
        for w in prog:
            op, fl, a, b = P.fields(int(w))
            k0 = k1 = -1
            if _arity(op) == 2:
                k1 = st.pop()
                k0 = st.pop()
            elif _arity(op) == 1:
                k0 = st.pop()
            inv = fl & 1 if op in P.ROLE_OPS else 0
            if not (op == P.ATOM or op in P.ROLE_OPS or op in P.DATA_OPS or op in P.STRING_OPS):
                a = 0
            if not (op in P.COUNT_OPS or op in P.DATA_OPS or op in P.STRING_OPS):
                b = 0
            self.nodes.append((op, inv, a, b, k0, k1))
            st.append(len(self.nodes) - 1)
        self.root = st[-1]
        n = len(self.nodes)
        mat = [False] * n
        for op, inv, a, b, k0, k1 in self.nodes:
            if op in P.ROLE_OPS and self.nodes[k0][0] != P.ATOM:
                mat[k0] = True
        need = [1] * n
        for i, (op, inv, a, b, k0, k1) in enumerate(self.nodes):
            nd = lambda c: 1 if mat[c] else need[c]
            if op == P.NOT:
                need[i] = nd(k0)
            elif op in (P.AND, P.OR):
                x, y = nd(k0), nd(k1)
                v = x + 1 if x == y else max(x, y)
                if v > STACK_MAX - 1:
                    mat[k0 if x >= y else k1] = True
                    x, y = nd(k0), nd(k1)
                    v = x + 1 if x == y else max(x, y)
                need[i] = v
        self.mat, self.need = mat, need
        self.mat_nodes = [i for i in range(n) if mat[i]]           # local slot j = mat_nodes[j]
        self.slot_of = {i: j for j, i in enumerate(self.mat_nodes)}
        self.kb = kb
        self.segs = [self._emit(i, True) for i in self.mat_nodes] + [self._emit(self.root, False)]
        # levels in node order: a materialised node's segment is one above the slots it reads
        slot_level = {}
        for j, i in enumerate(self.mat_nodes):
            s = self.segs[j]
            s["level"] = max((slot_level[r] + 1 for r in s["reads"]), default=0)
            slot_level[j] = s["level"]
        r = self.segs[-1]
        r["level"] = max((slot_level[x] + 1 for x in r["reads"]), default=0)

    def _emit(self, root: int, materialised: bool) -> dict:
        kb, nodes, mat = self.kb, self.nodes, self.mat
        code, reads = [], []
        rk, filler, model = NO_FILLER, NO_FILLER, 0
        N, B = kb["n"], 4 * kb["wp"]

        def visit(i: int):
            nonlocal rk, filler, model
            op, inv, a, b, k0, k1 = nodes[i]
            if i != root and mat[i]:
                code.append((D_SLOT, 0, 0, ("slot", self.slot_of[i])))
                reads.append(self.slot_of[i])
            elif op == P.ATOM:
                code.append((D_ATOM, a, 0, 0))
                model += B
            elif op in (P.TOP, P.BOT):
                code.append((op, 0, 0, 0))
            elif op in P.DATA_OPS:
                num = a >= kb["n_props"]
                code.append((D_DATA | (op << 16) | ((1 << 8) if num else 0), a - kb["n_props"] if num else a, b, 0))
                model += 4 * N if not num else 4 * (N + 1) + 4 * kb["num_vals"][a - kb["n_props"]]
            elif op in P.STRING_OPS:
                code.append((D_DATA | (op << 16) | (1 << 9), a, b, 0))
                model += 4 * (N + 1) + 4 * kb["str_vals"][a] + (4 * kb["contain_words"] if op == P.SCONTAINS else 0)
            elif op in P.ROLE_OPS:
                c = k0
                if nodes[c][0] == P.ATOM and not mat[c]:
                    ref = nodes[c][2]
                    model += B                      # the filler concept's row
                else:
                    ref = ("slot", self.slot_of[c])
                    reads.append(self.slot_of[c])
                code.append((D_ROLE | (inv << 8) | (op << 16), a, b, ref))
                if rk == NO_FILLER:
                    rk = a * 2 + inv
                if filler == NO_FILLER:
                    filler = ("filler", ref, REF_NEG if op == P.FORALL else 0)
                model += 4 * (N + 1) + 4 * kb["role_edges"][a] + 2 * B
            elif op == P.NOT:
                visit(k0)
                code.append((D_NOT, 0, 0, 0))
            else:   # AND / OR: the operand with the larger stack need first
                nd = lambda c: 1 if mat[c] else self.need[c]
                first = k0 if nd(k0) >= nd(k1) else k1
                visit(first)
                visit(k1 if first == k0 else k0)
                code.append((op, 0, 0, 0))

        visit(root)
        if not materialised:
            model += 2 * B + 16
        return {"code": code, "reads": sorted(set(reads)), "rk": rk, "filler": filler, "model": model}


def _align(x: int) -> int:
    return (x + 255) & ~255


def _put(img: bytearray, fmt: str, rows) -> int:
    off = _align(len(img))
    img.extend(b"\0" * (off - len(img)))
    for r in rows:
        img.extend(struct.pack(fmt, *r))
    return off


def plan_image(progs: Sequence[np.ndarray], kb: dict, flags: int, warps: int = 8, wpl: int = 1, rounds: int = 2,
               timeout_ms: int = 2000, n_sms: int = 152):
    """The image, the workspace bytes and the model bytes of the batch (steps 1-4)."""
    hyps = [Hyp(p, kb) for p in progs]
    H = len(hyps)
    # step 3: prefix sums over hypotheses
    slot_base, s = [], 0
    for h in hyps:
        slot_base.append(s)
        s += len(h.mat_nodes)
    n_slots = s
    segs = []                                   # (hyp index, local seg, out slot, hyp id)
    for hi, h in enumerate(hyps):
        for j in range(len(h.mat_nodes)):
            segs.append((hi, j, slot_base[hi] + j, NO_HYP))
    for hi, h in enumerate(hyps):
        segs.append((hi, len(h.segs) - 1, NO_SLOT, hi))
    gref = lambda hi, ref: (REF_SLOT | (slot_base[hi] + ref[1])) if isinstance(ref, tuple) else ref
    code, seg_rows, deps, levels, keys, model = [], [], [], [], [], 0
    walks = []
    for hi, j, out, hyp in segs:
        sg = hyps[hi].segs[j]
        c0 = len(code)
        for op, a, b, ref in sg["code"]:
            if op == D_SLOT:
                code.append((op, a, b, slot_base[hi] + ref[1]))
            else:
                code.append((op, a, b, gref(hi, ref)))
        d0 = len(deps)
        deps += [slot_base[hi] + r for r in sg["reads"]]   # the producer of slot g is segment g
        f = sg["filler"]
        filler = NO_FILLER if f == NO_FILLER else (gref(hi, f[1]) | f[2])
        seg_rows.append([c0, len(code) - c0, out, hyp, d0, len(deps) - d0, filler, 0])
        levels.append(sg["level"])
        keys.append(sg["rk"])
        walks.append(any((op & 0xFF) == D_ROLE for op, _, _, _ in sg["code"]))
        model += sg["model"]
    NS = len(segs)
    n_levels = max(levels) + 1
    # step 4: tile shape from the segments per level that walk a role
    wp = kb["wp"]
    WW, rnd = 32, rounds
    per_level = [0] * n_levels
    walk_level = [False] * n_levels
    for lv, w in zip(levels, walks):
        per_level[lv] += 1
        walk_level[lv] |= w
    smin = min((per_level[lv] for lv in range(n_levels) if walk_level[lv]), default=None)
    resident = 32 * n_sms
    if smin is not None:
        while WW > 4 and smin * wp < 4 * resident * WW * wpl:
            WW >>= 1
    if WW < 32:
        rnd = 1
    TW = warps * WW * wpl * rnd
    n_tiles = (wp + TW - 1) // TW
    order = sorted(range(NS), key=lambda x: (levels[x], keys[x]))      # stable
    groups, gsegs, level_items, items = [], [], [0] * (n_levels + 1), 0
    k = 0
    while k < NS:
        s0 = order[k]
        k2 = k
        start = len(gsegs)
        while k2 < NS and levels[order[k2]] == levels[s0] and keys[order[k2]] == keys[s0]:
            gsegs.append(order[k2])
            k2 += 1
        groups.append((items, start, k2 - k, levels[s0]))
        items += (k2 - k) * n_tiles
        level_items[levels[s0] + 1] = items
        k = k2
    for lv in range(1, n_levels + 1):
        level_items[lv] = max(level_items[lv], level_items[lv - 1])
    # the image
    img = bytearray(struct.calcsize(HEADER))
    off_segs = _put(img, SEG, seg_rows)
    off_groups = _put(img, GROUP, groups)
    off_gsegs = _put(img, "<I", [(x,) for x in gsegs])
    off_deps = _put(img, "<I", [(x,) for x in deps])
    off_code = _put(img, INSN, code)
    off_li = _put(img, "<I", [(x,) for x in level_items])
    off_ctr = _put(img, "<I", [(0,)] * (4 + NS + 1 + 2 * H))
    off_rg = _put(img, "<I", [])
    img.extend(b"\0" * (_align(len(img)) - len(img)))
    off_slots = len(img)
    off_ft = _align(off_slots + n_slots * 4 * wp)
    hdr = struct.pack(HEADER, items, NS, len(groups), H, n_tiles, TW, n_slots, flags, n_levels, len(deps), 0, WW,
                      off_segs, off_groups, off_gsegs, off_deps, off_code, off_li, off_ctr, off_slots, off_rg, off_ft,
                      timeout_ms * 1_000_000)
    img[:len(hdr)] = hdr
    return np.frombuffer(bytes(img), np.uint8), off_ft, model
