#!/usr/bin/env python3
"""Generates the per-angular-class ERI device code (Obara-Saika VRR + Head-Gordon-Pople HRR).

For every shell-quartet class (la lb | lc ld) with la >= lb, lc >= ld and the higher pair class on
the bra side, emit straight-line CUDA that, for one shell quartet,
  1. loops over primitive quartets: Boys F_m(T), m = 0..L, then the VRR
        [e+1_i,0|00]^(m) = PA_i [e0|00]^(m) + WP_i [e0|00]^(m+1)
                           + e_i/(2 zeta) ([e-1_i,0|00]^(m) - rho/zeta [e-1_i,0|00]^(m+1))
        [e0|f+1_i,0]^(m) = QC_i [e0|f0]^(m) + WQ_i [e0|f0]^(m+1)
                           + f_i/(2 eta) ([e0|f-1_i,0]^(m) - rho/eta [e0|f-1_i,0]^(m+1))
                           + e_i/(2(zeta+eta)) [e-1_i,0|f0]^(m+1)
     accumulating the contracted [e0|f0] for la <= |e| <= la+lb, lc <= |f| <= lc+ld;
  2. applies the HRR on the contracted sums,
        (a, b+1_i| = (a+1_i, b| + AB_i (a, b|,      |c, d+1_i) = |c+1_i, d) + CD_i |c, d);
  3. scales each Cartesian component by sqrt((2L-1)!! / ((2l-1)!!(2m-1)!!(2n-1)!!)), which turns
     the x^L-normalised contraction into per-component unit-norm functions.
Writes ``eri_class_<la><lb><lc><ld>.cuh`` files plus ``eri_classes.h`` (the class table) into the
output directory.  Run: ``gen_eri.py <outdir>``.
"""
from __future__ import annotations

import math
import os
import sys

import numpy as np

PAIR_CLASSES = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
QUARTET_CLASSES = [(PAIR_CLASSES[i], PAIR_CLASSES[j])
                   for i in range(len(PAIR_CLASSES)) for j in range(i + 1)]


def cart(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def ncart(l):
    return (l + 1) * (l + 2) // 2


def cidx(t):
    """index of Cartesian triple t within cart(sum(t))"""
    return cart(sum(t)).index(tuple(t))


def sub(v, i, k=1):
    w = list(v)
    w[i] -= k
    return tuple(w)


def add(v, i, k=1):
    w = list(v)
    w[i] += k
    return tuple(w)


def dfact(k):
    r = 1
    while k > 1:
        r *= k
        k -= 2
    return r


def comp_scale(t):
    L = sum(t)
    return math.sqrt(dfact(2 * L - 1) / (dfact(2 * t[0] - 1) * dfact(2 * t[1] - 1) * dfact(2 * t[2] - 1)))


def pick_dir(v):
    """direction used to lower a Cartesian triple: its largest component (ties: lowest axis)"""
    best = 0
    for i in range(3):
        if v[i] > v[best]:
            best = i
    return best


XYZ = "xyz"


class VRR:
    def __init__(self, la, lb, lc, ld):
        self.la, self.lb, self.lc, self.ld = la, lb, lc, ld
        self.L = la + lb + lc + ld
        self.order = []
        self.names = {}
        self.es = [e for E in range(la, la + lb + 1) for e in cart(E)]
        self.fs = [f for F in range(lc, lc + ld + 1) for f in cart(F)]
        for e in self.es:
            for f in self.fs:
                self._need(e, f, 0)

    def _need(self, e, f, m):
        key = (e, f, m)
        if key in self.names:
            return
        deps = []
        if sum(f) > 0:
            i = pick_dir(f)
            f1 = sub(f, i)
            deps = [(e, f1, m), (e, f1, m + 1)]
            if f1[i] >= 1:
                deps += [(e, sub(f1, i), m), (e, sub(f1, i), m + 1)]
            if e[i] >= 1:
                deps += [(sub(e, i), f1, m + 1)]
        elif sum(e) > 0:
            i = pick_dir(e)
            e1 = sub(e, i)
            deps = [(e1, f, m), (e1, f, m + 1)]
            if e1[i] >= 1:
                deps += [(sub(e1, i), f, m), (sub(e1, i), f, m + 1)]
        for d in deps:
            self._need(*d)
        self.names[key] = f"v{len(self.order)}"
        self.order.append(key)

    def emit(self, out, indent):
        flops = 0
        for (e, f, m) in self.order:
            nm = self.names[(e, f, m)]
            if sum(e) == 0 and sum(f) == 0:
                out.append(f"{indent}const R {nm} = F[{m}];")
                continue
            if sum(f) > 0:
                i = pick_dir(f)
                f1 = sub(f, i)
                x = XYZ[i]
                terms = f"QC{x} * {self.names[(e, f1, m)]} + WQ{x} * {self.names[(e, f1, m + 1)]}"
                flops += 3
                if f1[i] >= 1:
                    f2 = sub(f1, i)
                    terms += (f" + R({f1[i]}) * oo2e * ({self.names[(e, f2, m)]}"
                              f" - roe * {self.names[(e, f2, m + 1)]})")
                    flops += 4
                if e[i] >= 1:
                    terms += f" + R({e[i]}) * oo2ze * {self.names[(sub(e, i), f1, m + 1)]}"
                    flops += 3
            else:
                i = pick_dir(e)
                e1 = sub(e, i)
                x = XYZ[i]
                terms = f"PA{x} * {self.names[(e1, f, m)]} + WP{x} * {self.names[(e1, f, m + 1)]}"
                flops += 3
                if e1[i] >= 1:
                    e2 = sub(e1, i)
                    terms += (f" + R({e1[i]}) * oo2z * ({self.names[(e2, f, m)]}"
                              f" - roz * {self.names[(e2, f, m + 1)]})")
                    flops += 4
            out.append(f"{indent}const R {nm} = {terms};")
        return flops


def hrr_bra(la, lb, fs, es, out, indent, accname):
    """(a b| f] for a in cart(la), b in cart(lb), every f: from acc[e][f]. Returns (names, flops)."""
    nf = len(fs)
    eidx = {e: k for k, e in enumerate(es)}
    memo = {}
    counter = [0]
    flops = [0]

    def get(a, b, fi):
        key = (a, b, fi)
        if key in memo:
            return memo[key]
        if sum(b) == 0:
            nm = f"{accname}[{eidx[a] * nf + fi}]"
            memo[key] = nm
            return nm
        i = pick_dir(b)
        b1 = sub(b, i)
        t1 = get(add(a, i), b1, fi)
        t2 = get(a, b1, fi)
        nm = f"hb{counter[0]}"
        counter[0] += 1
        out.append(f"{indent}const R {nm} = {t1} + AB{XYZ[i]} * {t2};")
        flops[0] += 2
        memo[key] = nm
        return nm

    res = {}
    for fi in range(nf):
        for a in cart(la):
            for b in cart(lb):
                res[(a, b, fi)] = get(a, b, fi)
    return res, flops[0]


def hrr_ket(lc, ld, fs, brares, la, lb, out, indent):
    """(ab|cd) from (ab|f]."""
    fidx = {f: k for k, f in enumerate(fs)}
    memo = {}
    counter = [0]
    flops = [0]

    def get(ab, c, d):
        key = (ab, c, d)
        if key in memo:
            return memo[key]
        if sum(d) == 0:
            nm = brares[(ab[0], ab[1], fidx[c])]
            memo[key] = nm
            return nm
        i = pick_dir(d)
        d1 = sub(d, i)
        t1 = get(ab, add(c, i), d1)
        t2 = get(ab, c, d1)
        nm = f"hk{counter[0]}"
        counter[0] += 1
        out.append(f"{indent}const R {nm} = {t1} + CD{XYZ[i]} * {t2};")
        flops[0] += 2
        memo[key] = nm
        return nm

    res = {}
    for a in cart(la):
        for b in cart(lb):
            for c in cart(lc):
                for d in cart(ld):
                    res[(a, b, c, d)] = get((a, b), c, d)
    return res, flops[0]


# ------------------------------------------------------------------------------------------------
# Op programs for the generic (interpreted) kernel.  The VRR / HRR sequences are the same as in the
# straight-line code; slots are assigned by a linear scan over live intervals so that the per-thread
# working arrays only hold the values that are live at the same time.
# ------------------------------------------------------------------------------------------------
def _linear_scan(n_values, defs_uses, pinned=()):
    """defs_uses: list over op positions of (defined_value or None, [used values]).
    Returns slot per value and the number of slots."""
    last = {}
    for pos, (d, uses) in enumerate(defs_uses):
        for u in uses:
            last[u] = pos
    for v in pinned:
        last[v] = len(defs_uses)
    free = []
    nslots = 0
    slot = {}
    for pos, (d, uses) in enumerate(defs_uses):
        # release values whose last use is this op (after reading them)
        if d is not None:
            # allocate before releasing so the target never aliases a source of the same op
            if free:
                slot[d] = free.pop()
            else:
                slot[d] = nslots
                nslots += 1
            if d not in last:
                last[d] = pos
        for u in set(uses):
            if last.get(u) == pos:
                free.append(slot[u])
        if d is not None and last[d] == pos and d not in pinned:
            free.append(slot[d])
    return slot, nslots


def check_program(pr, nvi=None):
    """Every slot an op program names lies inside the arrays the kernels declare for it (V: nvi
    slots, default nv; H: nh slots), the contracted values fill H's first nacc slots, the base
    values read F[m] with m <= L, and every field fits its bit width in the encoded words."""
    nv, nh, nacc, L = pr["nv"], pr["nh"], pr["nacc"], pr["L"]
    nvi = nv if nvi is None else nvi
    assert nacc <= nh and nv <= nvi, (nacc, nh, nv, nvi)
    assert nvi < 1 << 16 and nh < 1 << 16
    for (kind, t, s1, s2, s3, s4, s5, d, m1, m2) in pr["vrr"]:
        assert 0 <= t < nv and 0 <= d < 3 and 0 <= m1 < 16 and 0 <= m2 < 16
        if kind == 0:
            assert 0 <= s1 <= L
        elif kind == 3:
            assert 0 <= s1 < nacc
        else:
            assert kind in (1, 2) and all(0 <= x < nv for x in (s1, s2, s3, s4, s5))
    for (t, s1, s2, d, side) in pr["hrr"]:
        assert 0 <= t < nh and 0 <= s1 < nh and 0 <= s2 < nh and 0 <= d < 3 and side in (0, 1)
    assert len(pr["fin"]) == pr["na"] * pr["nb"] * pr["nc"] * pr["nd"]
    assert all(0 <= f < nh for f, _ in pr["fin"])
    return pr


def build_program(cls):
    (la, lb), (lc, ld) = cls
    v = VRR(la, lb, lc, ld)
    nf = len(v.fs)
    accidx = {}
    for ei, e in enumerate(v.es):
        for fi, f in enumerate(v.fs):
            accidx[(e, f, 0)] = ei * nf + fi
    # VRR ops: (kind, target, s1, s2, s3, s4, s5, dir, m1, m2); kind 0 base, 1 bra, 2 ket, 3 acc
    raw = []
    for key in v.order:
        e, f, m = key
        if sum(e) == 0 and sum(f) == 0:
            raw.append((0, key, [], m, 0, 0, 0))
        elif sum(f) > 0:
            i = pick_dir(f)
            f1 = sub(f, i)
            srcs = [(e, f1, m), (e, f1, m + 1)]
            m1 = f1[i]
            srcs += [(e, sub(f1, i), m), (e, sub(f1, i), m + 1)] if m1 >= 1 else [None, None]
            m2 = e[i]
            srcs += [(sub(e, i), f1, m + 1)] if m2 >= 1 else [None]
            raw.append((2, key, srcs, None, i, m1, m2))
        else:
            i = pick_dir(e)
            e1 = sub(e, i)
            srcs = [(e1, f, m), (e1, f, m + 1)]
            m1 = e1[i]
            srcs += [(sub(e1, i), f, m), (sub(e1, i), f, m + 1)] if m1 >= 1 else [None, None]
            srcs += [None]
            raw.append((1, key, srcs, None, i, m1, 0))
        if key in accidx:
            raw.append((3, key, [key], accidx[key], 0, 0, 0))
    du = []
    for (kind, key, srcs, extra, d, m1, m2) in raw:
        uses = [x for x in srcs if x is not None]
        du.append((key if kind != 3 else None, uses))
    slot, nv = _linear_scan(len(v.order), du)
    vrr_ops = []
    for (kind, key, srcs, extra, d, m1, m2) in raw:
        if kind == 0:
            vrr_ops.append((0, slot[key], extra, 0, 0, 0, 0, 0, 0, 0))
        elif kind == 3:
            vrr_ops.append((3, slot[key], extra, 0, 0, 0, 0, 0, 0, 0))
        else:
            ss = [slot[x] if x is not None else 0 for x in srcs]
            vrr_ops.append((kind, slot[key], ss[0], ss[1], ss[2], ss[3], ss[4], d, m1, m2))
    # HRR ops on H: values 'acc k' first (pinned into slots 0..nacc-1), then bra/ket intermediates
    nacc = len(v.es) * nf
    eidx = {e: k for k, e in enumerate(v.es)}
    fidx = {f: k for k, f in enumerate(v.fs)}
    hops = []          # (target value, src1 value, src2 value, dir, side)
    memo_b = {}

    def gb(a, b, fi):
        key = ("b", a, b, fi)
        if key in memo_b:
            return memo_b[key]
        if sum(b) == 0:
            val = ("acc", eidx[a] * nf + fi)
        else:
            i = pick_dir(b)
            b1 = sub(b, i)
            t1 = gb(add(a, i), b1, fi)
            t2 = gb(a, b1, fi)
            val = key
            hops.append((val, t1, t2, i, 0))
        memo_b[key] = val
        return val
    memo_k = {}

    def gk(a, b, c, d):
        key = ("k", a, b, c, d)
        if key in memo_k:
            return memo_k[key]
        if sum(d) == 0:
            val = gb(a, b, fidx[c])
        else:
            i = pick_dir(d)
            d1 = sub(d, i)
            t1 = gk(a, b, add(c, i), d1)
            t2 = gk(a, b, c, d1)
            val = key
            hops.append((val, t1, t2, i, 1))
        memo_k[key] = val
        return val
    finals = []
    for a in cart(la):
        for b in cart(lb):
            for c in cart(lc):
                for d in cart(ld):
                    finals.append((gk(a, b, c, d), comp_scale(a) * comp_scale(b) * comp_scale(c) * comp_scale(d)))
    # slot allocation for H: acc values pinned at 0..nacc-1 until their last use, finals pinned to the end
    du = [(None, [])]  # position 0: all acc values defined (pre-existing)
    for (t, s1, s2, d, side) in hops:
        du.append((t, [s1, s2]))
    final_vals = [f for f, _ in finals]
    # custom scan: acc values occupy fixed slots; other values get slots >= nacc
    last = {}
    for pos, (d, uses) in enumerate(du):
        for u in uses:
            last[u] = pos
    for fv in final_vals:
        last[fv] = len(du)
    hslot = {("acc", k): k for k in range(nacc)}
    free = []
    nh = nacc
    for pos, (d, uses) in enumerate(du):
        if d is not None:
            if free:
                hslot[d] = free.pop()
            else:
                hslot[d] = nh
                nh += 1
        for u in set(uses):
            if last.get(u) == pos:
                free.append(hslot[u])
    hrr_ops = [(hslot[t], hslot[s1], hslot[s2], d, side) for (t, s1, s2, d, side) in hops]
    fin = [(hslot[fv], sc) for fv, sc in finals]
    return check_program(dict(vrr=vrr_ops, nv=nv, hrr=hrr_ops, nh=nh, fin=fin, nacc=nacc, L=la + lb + lc + ld,
                              na=ncart(la), nb=ncart(lb), nc=ncart(lc), nd=ncart(ld)))


def _level_alloc(values, deflev, lastlev, pinned_slots=None, pinned_end=()):
    """Slots for level-parallel execution: a value occupies its slot from its defining level
    through its last-use level; a slot is reused only by a value defined at a later level."""
    for v in pinned_end:
        lastlev[v] = 10 ** 9
    slot = dict(pinned_slots or {})
    nslots = max(slot.values()) + 1 if slot else 0
    busy_until = {sl: lastlev[v] for v, sl in slot.items()}   # slot -> last level it is read
    order = sorted((v for v in values if v not in slot), key=lambda v: deflev[v])
    free = []
    for v in order:
        L = deflev[v]
        # release slots whose occupant was last read before level L
        for sl, until in list(busy_until.items()):
            if until < L:
                free.append(sl)
                del busy_until[sl]
        if free:
            free.sort()
            sl = free.pop(0)
        else:
            sl = nslots
            nslots += 1
        slot[v] = sl
        busy_until[sl] = lastlev.get(v, L)
    return slot, nslots


def build_team_program(cls):
    """Level-scheduled op program for one warp per shell quartet (lanes run the independent ops of
    one dependency level in parallel; values in shared memory)."""
    (la, lb), (lc, ld) = cls
    v = VRR(la, lb, lc, ld)
    nf = len(v.fs)
    accidx = {}
    for ei, e in enumerate(v.es):
        for fi, f in enumerate(v.fs):
            accidx[(e, f, 0)] = ei * nf + fi
    lev, deps = {}, {}
    meta = {}
    for key in v.order:
        e, f, m = key
        if sum(e) == 0 and sum(f) == 0:
            d, info = [], (0, [], m, 0, 0, 0)
        elif sum(f) > 0:
            i = pick_dir(f)
            f1 = sub(f, i)
            srcs = [(e, f1, m), (e, f1, m + 1)]
            m1 = f1[i]
            srcs += [(e, sub(f1, i), m), (e, sub(f1, i), m + 1)] if m1 >= 1 else [None, None]
            m2 = e[i]
            srcs += [(sub(e, i), f1, m + 1)] if m2 >= 1 else [None]
            d, info = [x for x in srcs if x is not None], (2, srcs, None, i, m1, m2)
        else:
            i = pick_dir(e)
            e1 = sub(e, i)
            srcs = [(e1, f, m), (e1, f, m + 1)]
            m1 = e1[i]
            srcs += [(sub(e1, i), f, m), (sub(e1, i), f, m + 1)] if m1 >= 1 else [None, None]
            srcs += [None]
            d, info = [x for x in srcs if x is not None], (1, srcs, None, i, m1, 0)
        lev[key] = 1 + max([lev[x] for x in d], default=-1)
        deps[key] = d
        meta[key] = info
    # ACC ops one level after their value
    lastv = {}
    for key in v.order:
        for x in deps[key]:
            lastv[x] = max(lastv.get(x, -1), lev[key])
    for key in accidx:
        lastv[key] = max(lastv.get(key, -1), lev[key] + 1)
    vslot, nv = _level_alloc(list(v.order), lev, lastv)
    nlev = max(lev.values()) + 2
    ops_by_level = [[] for _ in range(nlev)]
    for key in v.order:
        kind, srcs, m, d, m1, m2 = meta[key]
        if kind == 0:
            ops_by_level[lev[key]].append((0, vslot[key], m, 0, 0, 0, 0, 0, 0, 0))
        else:
            ss = [vslot[x] if x is not None else 0 for x in srcs]
            ops_by_level[lev[key]].append((kind, vslot[key], ss[0], ss[1], ss[2], ss[3], ss[4], d, m1, m2))
    for key, k in accidx.items():
        ops_by_level[lev[key] + 1].append((3, vslot[key], k, 0, 0, 0, 0, 0, 0, 0))
    ops_by_level = [l for l in ops_by_level if l]
    vops, vlev = [], [0]
    for l in ops_by_level:
        vops += l
        vlev.append(len(vops))
    # HRR: same value graph as build_program, scheduled by levels
    eidx = {e: k for k, e in enumerate(v.es)}
    fidx = {f: k for k, f in enumerate(v.fs)}
    hops, hlevel = [], {}
    memo_b, memo_k = {}, {}

    def gb(a, b, fi):
        key = ("b", a, b, fi)
        if key in memo_b:
            return memo_b[key]
        if sum(b) == 0:
            val = ("acc", eidx[a] * nf + fi)
            hlevel[val] = 0
        else:
            i = pick_dir(b)
            b1 = sub(b, i)
            t1, t2 = gb(add(a, i), b1, fi), gb(a, b1, fi)
            val = key
            hlevel[val] = 1 + max(hlevel[t1], hlevel[t2])
            hops.append((val, t1, t2, i, 0))
        memo_b[key] = val
        return val

    def gk(a, b, c, dd):
        key = ("k", a, b, c, dd)
        if key in memo_k:
            return memo_k[key]
        if sum(dd) == 0:
            val = gb(a, b, fidx[c])
        else:
            i = pick_dir(dd)
            d1 = sub(dd, i)
            t1, t2 = gk(a, b, add(c, i), d1), gk(a, b, c, d1)
            val = key
            hlevel[val] = 1 + max(hlevel[t1], hlevel[t2])
            hops.append((val, t1, t2, i, 1))
        memo_k[key] = val
        return val
    finals = []
    for a in cart(la):
        for b in cart(lb):
            for c in cart(lc):
                for dd in cart(ld):
                    finals.append((gk(a, b, c, dd), comp_scale(a) * comp_scale(b) * comp_scale(c) * comp_scale(dd)))
    nacc = len(v.es) * nf
    lasth = {}
    for (t, s1, s2, d, side) in hops:
        for x in (s1, s2):
            lasth[x] = max(lasth.get(x, 0), hlevel[t])
    for k in range(nacc):
        lasth.setdefault(("acc", k), 0)
    pinned = {("acc", k): k for k in range(nacc)}
    values = [h[0] for h in hops]
    hslot, nh = _level_alloc(values, hlevel, lasth, pinned, pinned_end=[f for f, _ in finals])
    nhl = max([hlevel[h[0]] for h in hops], default=0)
    hops_by_level = [[] for _ in range(nhl + 1)]
    for (t, s1, s2, d, side) in hops:
        hops_by_level[hlevel[t]].append((hslot[t], hslot[s1], hslot[s2], d, side))
    hops_by_level = [l for l in hops_by_level if l]
    hprog, hlev = [], [0]
    for l in hops_by_level:
        hprog += l
        hlev.append(len(hprog))
    fin = [(hslot[f], sc) for f, sc in finals]
    nint = len(fin)
    pr = dict(vrr=vops, vlev=vlev, nv=nv, hrr=hprog, hlev=hlev, nh=nh, fin=fin, nacc=nacc,
              L=la + lb + lc + ld, nint=nint, na=ncart(la), nb=ncart(lb), nc=ncart(lc), nd=ncart(ld))
    # the warp/block kernels store the final integrals over the V region: nvi = max(nv, nint) slots
    return check_program(pr, nvi=max(nv, nint))


# straight-line classes with at most this many VRR entries unroll their FP32 primitive loop by two
PRIM_UNROLL_MAX_VRR = 24


def straight_line(info):
    """classes emitted as straight-line register code (the rest run the op-program kernel)"""
    return info["nacc"] <= 96 and info["nvrr"] <= 280


def tag(cls):
    (la, lb), (lc, ld) = cls
    return f"{la}{lb}{lc}{ld}"


def emit_class_straight(cls):
    (la, lb), (lc, ld) = cls
    t = tag(cls)
    L = la + lb + lc + ld
    v = VRR(la, lb, lc, ld)
    na, nb, nc, nd = ncart(la), ncart(lb), ncart(lc), ncart(ld)
    nint = na * nb * nc * nd
    nacc = len(v.es) * len(v.fs)
    lines = []
    lines.append(f"// ---- class ({la}{lb}|{lc}{ld}): {len(v.order)} VRR entries, {nacc} contracted, {nint} integrals")
    lines.append(f"template <typename R, int BMODE, int G>")
    lines.append(f"__device__ __forceinline__ void eri_{t}(const PairTable<R>& P, int bp, const KetView<R>& kv, int g, R* I, bool live = true)")
    lines.append("{")
    lines.append(f"    R acc[{nacc}];")
    lines.append(f"#pragma unroll")
    lines.append(f"    for (int k = 0; k < {nacc}; ++k) acc[k] = R(0);")
    lines.append("    const int k0 = kv.k0, nk = kv.nk, k1 = k0 + nk;")
    lines.append("    // !live, or a ket without primitives: no primitive work")
    lines.append("    const int b0 = P.pp_off[bp], b1 = b0 + ((live && nk > 0) ? P.pp_n[bp] : 0);")
    lines.append("    // A - C in FP64, then P - Q = (P - A) - (Q - C) + (A - C): no absolute coordinates in R")
    lines.append("    const R ACx = kv.AC[0], ACy = kv.AC[1], ACz = kv.AC[2];")
    body = []
    body.append("            R rz, srz;")
    body.append("            recip_and_sqrt(pb.zeta + pk.zeta, rz, srz);")
    body.append("            const R roz = pk.zeta * rz, roe = pb.zeta * rz, oo2ze = R(0.5) * rz;")
    body.append("            const R oo2z = pb.oo2z, oo2e = pk.oo2z;")
    body.append("            (void)roe; (void)roz; (void)oo2ze; (void)oo2z; (void)oo2e;")
    body.append("            const R PQx = pb.PAx - pk.PAx + ACx, PQy = pb.PAy - pk.PAy + ACy, PQz = pb.PAz - pk.PAz + ACz;")
    body.append("            const R PAx = pb.PAx, PAy = pb.PAy, PAz = pb.PAz;")
    body.append("            const R QCx = pk.PAx, QCy = pk.PAy, QCz = pk.PAz;")
    body.append("            const R WPx = -roz * PQx, WPy = -roz * PQy, WPz = -roz * PQz;")
    body.append("            const R WQx = roe * PQx, WQy = roe * PQy, WQz = roe * PQz;")
    body.append("            (void)PAx; (void)PAy; (void)PAz; (void)QCx; (void)QCy; (void)QCz;")
    body.append("            (void)WPx; (void)WPy; (void)WPz; (void)WQx; (void)WQy; (void)WQz;")
    body.append("            const R T = pb.zeta * roz * (PQx * PQx + PQy * PQy + PQz * PQz);")
    body.append("            const R pref = pb.K * pk.K * srz;")
    body.append(f"            R F[{L + 1}];")
    body.append(f"            boys_eval<R, {L}, BMODE>(T, F, P);")
    body.append("#pragma unroll")
    body.append(f"            for (int m = 0; m <= {L}; ++m) F[m] *= pref;")
    vflops = v.emit(body, "            ")
    for ei, e in enumerate(v.es):
        for fi, f in enumerate(v.fs):
            body.append(f"            acc[{ei * len(v.fs) + fi}] += {v.names[(e, f, 0)]};")
    lines.append("    if constexpr (G == 1) {")
    lines.append("    // ket primitives outside: each lane's ket records (different for every lane) are read once;")
    lines.append("    // the bra records inside are the same for the whole warp (one broadcast load each)")
    lines.append("    const int k1l = live ? k1 : k0;")
    lines.append("#pragma unroll 1")
    lines.append("    for (int ik = k0; ik < k1l; ++ik) {")
    lines.append("        const PrimPair<R> pk = P.load(ik);")
    lines.append(f"#pragma unroll ({'PrimUnroll<R>::value' if len(v.order) <= PRIM_UNROLL_MAX_VRR else 1})")
    lines.append("        for (int ib = b0; ib < b1; ++ib) {")
    lines.append("            const PrimPair<R> pb = P.load(ib);")
    lines += body
    lines.append("        }")
    lines.append("    }")
    lines.append("    } else {")
    lines.append("    // the G lanes of a group split the primitive quartets (flattened index g, g + G, ...)")
    lines.append("    int ib = b0, ik = k0 + g;")
    lines.append("    while (ik >= k1 && ib < b1) { ik -= nk; ++ib; }")
    lines.append("#pragma unroll 1")
    lines.append("    while (ib < b1) {")
    lines.append("        {")
    lines.append("            const PrimPair<R> pb = P.load(ib);")
    lines.append("            const PrimPair<R> pk = P.load(ik);")
    lines += body
    lines.append("        }")
    lines.append("        ik += G;")
    lines.append("        while (ik >= k1 && ib < b1) { ik -= nk; ++ib; }")
    lines.append("    }")
    lines.append("#pragma unroll")
    lines.append(f"    for (int k = 0; k < {nacc}; ++k) acc[k] = group_sum<G>(acc[k]);")
    lines.append("    }")
    lines.append("    const R ABx = pair_ab(P, bp, 0), ABy = pair_ab(P, bp, 1), ABz = pair_ab(P, bp, 2);")
    lines.append("    const R CDx = kv.CD[0], CDy = kv.CD[1], CDz = kv.CD[2];")
    lines.append("    (void)ABx; (void)ABy; (void)ABz; (void)CDx; (void)CDy; (void)CDz;")
    hb, hbf = hrr_bra(la, lb, v.fs, v.es, lines, "    ", "acc")
    hk, hkf = hrr_ket(lc, ld, v.fs, hb, la, lb, lines, "    ")
    k = 0
    for a in cart(la):
        for b in cart(lb):
            for c in cart(lc):
                for d in cart(ld):
                    s = comp_scale(a) * comp_scale(b) * comp_scale(c) * comp_scale(d)
                    if abs(s - 1.0) < 1e-15:
                        lines.append(f"    I[{k}] = {hk[(a, b, c, d)]};")
                    else:
                        lines.append(f"    I[{k}] = R({s!r}) * {hk[(a, b, c, d)]};")
                    k += 1
    lines.append("}")
    info = dict(tag=t, la=la, lb=lb, lc=lc, ld=ld, L=L, nvrr=len(v.order), vrr_flops=vflops,
                hrr_flops=hbf + hkf, nacc=nacc, nint=nint)
    return "\n".join(lines) + "\n", info


def df32_program(info):
    """straight-line classes whose double-float quartets, one thread per quartet, run the op-program
    interpreter: double-float takes about ten FP32 instructions per operation, and the straight-line
    code of these classes would then overflow the instruction cache (the warps stall on fetch)"""
    return info["mode"] == "straight" and info["vrr_flops"] + info["hrr_flops"] >= 250


def emit_class(cls):
    body, info = emit_class_straight(cls)
    (la, lb), (lc, ld) = cls
    t = tag(cls)
    if straight_line(info):
        info["mode"] = "straight"
        if not df32_program(info):
            return body, info
        # straight-line code for every arithmetic but double-float with one thread per quartet
        pr = build_program(cls)
        body = body.replace(f"__device__ __forceinline__ void eri_{t}(", f"__device__ __forceinline__ void eri_{t}_sl(", 1)
        L = [body, f"// double-float, one thread per quartet: op program, {len(pr['vrr'])} VRR ops on {pr['nv']} "
                   f"slots, {len(pr['hrr'])} HRR ops on {pr['nh']} slots"]
        L += emit_program_tables(t, pr)
        L.append("template <typename R, int BMODE, int G>")
        L.append(f"__device__ __forceinline__ void eri_{t}(const PairTable<R>& P, int bp, const KetView<R>& kv, int g, R* I, bool live = true)")
        L.append("{")
        L.append("    if constexpr (std::is_same<R, df32>::value && G == 1) {")
        L.append("        (void)g;")
        L.append(f"        eri_program<R, BMODE, {pr['L']}, {pr['nv']}, {pr['nh']}, {pr['nacc']}, {len(pr['vrr'])}, "
                 f"{len(pr['hrr'])}, {len(pr['fin'])}>(P, bp, kv, vprog_{t}, hprog_{t}, fslot_{t}, fscale_{t}, "
                 f"fscaleh_{t}, fscalel_{t}, I, live);")
        L.append("    } else {")
        L.append(f"        eri_{t}_sl<R, BMODE, G>(P, bp, kv, g, I, live);")
        L.append("    }")
        L.append("}")
        return "\n".join(L) + "\n", info
    pr = build_program(cls)
    info["mode"] = "program"
    info["nv_slots"], info["nh_slots"] = pr["nv"], pr["nh"]
    L = []
    L.append(f"// ---- class ({la}{lb}|{lc}{ld}): op program, {len(pr['vrr'])} VRR ops on {pr['nv']} slots, "
             f"{len(pr['hrr'])} HRR ops on {pr['nh']} slots")
    L += emit_program_tables(t, pr)
    L.append("template <typename R, int BMODE, int G>")
    L.append(f"__device__ __forceinline__ void eri_{t}(const PairTable<R>& P, int bp, const KetView<R>& kv, int g, R* I, bool live = true)")
    L.append("{")
    L.append("    static_assert(G == 1, \"op-program classes run one thread per quartet\");")
    L.append("    (void)g;")
    L.append(f"    eri_program<R, BMODE, {pr['L']}, {pr['nv']}, {pr['nh']}, {pr['nacc']}, {len(pr['vrr'])}, "
             f"{len(pr['hrr'])}, {len(pr['fin'])}>(P, bp, kv, vprog_{t}, hprog_{t}, fslot_{t}, fscale_{t}, "
             f"fscaleh_{t}, fscalel_{t}, I, live);")
    L.append("}")
    return "\n".join(L) + "\n", info


def emit_program_tables(t, pr):
    """device tables of one op program (VRR and HRR op words, output slots and scales)"""
    L = []
    L.append(f"__device__ const uint4 vprog_{t}[{len(pr['vrr'])}] = {{")
    for (kind, tg, s1, s2, s3, s4, s5, d, m1, m2) in pr["vrr"]:
        w0 = kind | (d << 2) | (m1 << 4) | (m2 << 8) | (tg << 16)
        L.append(f"    {{{w0}u, {s1 | (s2 << 16)}u, {s3 | (s4 << 16)}u, {s5}u}},")
    L.append("};")
    L.append(f"__device__ const uint2 hprog_{t}[{max(1, len(pr['hrr']))}] = {{")
    for (tg, s1, s2, d, side) in pr["hrr"]:
        L.append(f"    {{{tg | (d << 16) | (side << 18)}u, {s1 | (s2 << 16)}u}},")
    if not pr["hrr"]:
        L.append("    {0u, 0u},")
    L.append("};")
    L.append(f"__device__ const int fslot_{t}[{len(pr['fin'])}] = {{" + ", ".join(str(a) for a, _ in pr["fin"]) + "};")
    L.append(f"__device__ const double fscale_{t}[{len(pr['fin'])}] = {{" + ", ".join(repr(b) for _, b in pr["fin"]) + "};")
    his = [float(np.float32(b)) for _, b in pr["fin"]]
    los = [float(np.float32(b - h)) for (_, b), h in zip(pr["fin"], his)]
    L.append(f"__device__ const float fscaleh_{t}[{len(pr['fin'])}] = {{" + ", ".join(repr(h) + "f" for h in his) + "};")
    L.append(f"__device__ const float fscalel_{t}[{len(pr['fin'])}] = {{" + ", ".join(repr(l) + "f" for l in los) + "};")
    return L


def emit_team(cls, info):
    """Level-scheduled program arrays + kernel arguments of the warp-per-quartet kernel."""
    t = tag(cls)
    L = []
    tp = build_team_program(cls)
    info["team_nvi"], info["team_nh"] = max(tp["nv"], tp["nint"]), tp["nh"]
    L.append(f"// level-scheduled program for the warp-per-quartet J/K kernel: {len(tp['vlev']) - 1} VRR levels, "
             f"{len(tp['hlev']) - 1} HRR levels, {tp['nv']} + {tp['nh']} shared-memory slots")
    L.append(f"__device__ const uint4 tvprog_{t}[{len(tp['vrr'])}] = {{")
    for (kind, tg, s1, s2, s3, s4, s5, d, m1, m2) in tp["vrr"]:
        w0 = kind | (d << 2) | (m1 << 4) | (m2 << 8) | (tg << 16)
        L.append(f"    {{{w0}u, {s1 | (s2 << 16)}u, {s3 | (s4 << 16)}u, {s5}u}},")
    L.append("};")
    L.append(f"__device__ const int tvlev_{t}[{len(tp['vlev'])}] = {{" + ", ".join(map(str, tp["vlev"])) + "};")
    L.append(f"__device__ const uint2 thprog_{t}[{max(1, len(tp['hrr']))}] = {{")
    for (tg, s1, s2, d, side) in tp["hrr"]:
        L.append(f"    {{{tg | (d << 16) | (side << 18)}u, {s1 | (s2 << 16)}u}},")
    if not tp["hrr"]:
        L.append("    {0u, 0u},")
    L.append("};")
    L.append(f"__device__ const int thlev_{t}[{len(tp['hlev'])}] = {{" + ", ".join(map(str, tp["hlev"])) + "};")
    L.append(f"__device__ const int tfslot_{t}[{len(tp['fin'])}] = {{" + ", ".join(str(a) for a, _ in tp["fin"]) + "};")
    L.append(f"__device__ const double tfscale_{t}[{len(tp['fin'])}] = {{" + ", ".join(repr(b) for _, b in tp["fin"]) + "};")
    his = [float(np.float32(b)) for _, b in tp["fin"]]
    los = [float(np.float32(b - h)) for (_, b), h in zip(tp["fin"], his)]
    L.append(f"__device__ const float tfscaleh_{t}[{len(tp['fin'])}] = {{" + ", ".join(repr(h) + "f" for h in his) + "};")
    L.append(f"__device__ const float tfscalel_{t}[{len(tp['fin'])}] = {{" + ", ".join(repr(l) + "f" for l in los) + "};")
    L.append(f"#define MESS_TEAM_ARGS_{t} {tp['L']}, {max(tp['nv'], tp['nint'])}, {tp['nh']}, {tp['nacc']}, "
             f"{len(tp['vlev']) - 1}, {len(tp['hlev']) - 1}, {tp['nint']}, {tp['na']}, {tp['nb']}, {tp['nc']}, {tp['nd']}")
    L.append(f"#define MESS_TEAM_PROG_{t} tvprog_{t}, tvlev_{t}, thprog_{t}, thlev_{t}, tfslot_{t}, tfscale_{t}, "
             f"tfscaleh_{t}, tfscalel_{t}")
    return "\n".join(L) + "\n"


def team_capable(info):
    """classes that get a warp-per-quartet kernel (always used for the op-program classes; used for
    the FP64 parts of the others)"""
    return info["nvrr"] >= 40


def emit_digests(cls, info):
    """The digestion of a class as the kernels call it (digest_<class>).  Straight-line classes stage
    the density blocks in registers; the op-program classes, and the double-float path of the
    straight-line classes that run the interpreter (df32_program), read D through the read-only
    cache: a one-thread kernel that inlines the interpreter must not also stage density arrays."""
    t = tag(cls)
    if info["mode"] != "straight":
        return emit_digest(cls, unroll=False)
    if not df32_program(info):
        return emit_digest(cls, unroll=True)
    return (emit_digest(cls, unroll=True, name=f"digest_{t}_st") + "\n"
            + emit_digest(cls, unroll=False, name=f"digest_{t}_ro") + "\n"
            + "template <typename R>\n"
            + f"__device__ __forceinline__ void digest_{t}(const R* I, const DigestCtx<R>& c, R s)\n"
            + "{\n"
            + f"    if constexpr (std::is_same<R, df32>::value) digest_{t}_ro<R>(I, c, s);\n"
            + f"    else digest_{t}_st<R>(I, c, s);\n"
            + "}\n")


def emit_digest(cls, unroll=True, name=None):
    """J/K digestion of one shell quartet (see the kernel file for the accumulation convention).
    unroll=True: density blocks staged in registers, loops fully unrolled (small classes);
    unroll=False: compact loops reading the density through the read-only cache (large classes)."""
    (la, lb), (lc, ld) = cls
    t = tag(cls)
    na, nb, nc, nd = ncart(la), ncart(lb), ncart(lc), ncart(ld)
    PR = "#pragma unroll" if unroll else "#pragma unroll 1"
    L = []
    L.append(f"template <typename R>")
    L.append(f"__device__ __forceinline__ void {name or 'digest_' + t}(const R* I, const DigestCtx<R>& c, R s)")
    L.append("{")
    blocks = (("Dab", ("c.fa", na), ("c.fb", nb)), ("Dcd", ("c.fc", nc), ("c.fd", nd)),
              ("Dac", ("c.fa", na), ("c.fc", nc)), ("Dad", ("c.fa", na), ("c.fd", nd)),
              ("Dbc", ("c.fb", nb), ("c.fc", nc)), ("Dbd", ("c.fb", nb), ("c.fd", nd)))
    dref = {}
    for nm, (r0, nr), (c0, ncol) in blocks:
        if unroll:
            L.append(f"    R {nm}[{nr * ncol}];")
            L.append(PR)
            L.append(f"    for (int i = 0; i < {nr}; ++i)")
            L.append(PR)
            L.append(f"        for (int j = 0; j < {ncol}; ++j) {nm}[i * {ncol} + j] = ldD(c.D + (size_t)({r0} + i) * c.n + {c0} + j);")
            dref[nm] = lambda a, b, nm=nm, ncol=ncol: f"{nm}[{a} * {ncol} + {b}]"
        else:
            dref[nm] = lambda a, b, r0=r0, c0=c0: f"ldD(c.D + (size_t)({r0} + {a}) * c.n + {c0} + {b})"
    I = f"I[((i * {nb} + j) * {nc} + k) * {nd} + l]"
    # J_ab
    L += [PR, f"    for (int i = 0; i < {na}; ++i)", PR, f"        for (int j = 0; j < {nb}; ++j) {{",
          "            R t = R(0);", PR, f"            for (int k = 0; k < {nc}; ++k)", PR,
          f"                for (int l = 0; l < {nd}; ++l) t += {I} * {dref['Dcd']('k', 'l')};",
          "            jk_add(c.J, (size_t)(c.fa + i) * c.n + c.fb + j, s * t, c.warp_reduce_ab);", "        }"]
    # J_cd
    L += [PR, f"    for (int k = 0; k < {nc}; ++k)", PR, f"        for (int l = 0; l < {nd}; ++l) {{",
          "            R t = R(0);", PR, f"            for (int i = 0; i < {na}; ++i)", PR,
          f"                for (int j = 0; j < {nb}; ++j) t += {I} * {dref['Dab']('i', 'j')};",
          "            jk_add(c.J, (size_t)(c.fc + k) * c.n + c.fd + l, s * t, false);", "        }"]
    # K blocks: K_ac (sum b,d D_bd), K_ad (sum b,c D_bc), K_bc (sum a,d D_ad), K_bd (sum a,c D_ac)
    for (o1, n1, f1), (o2, n2, f2), (s1, m1), (s2, m2), Dn in (
            (("i", na, "c.fa"), ("k", nc, "c.fc"), ("j", nb), ("l", nd), "Dbd"),
            (("i", na, "c.fa"), ("l", nd, "c.fd"), ("j", nb), ("k", nc), "Dbc"),
            (("j", nb, "c.fb"), ("k", nc, "c.fc"), ("i", na), ("l", nd), "Dad"),
            (("j", nb, "c.fb"), ("l", nd, "c.fd"), ("i", na), ("k", nc), "Dac")):
        L += [PR, f"    for (int {o1} = 0; {o1} < {n1}; ++{o1})", PR,
              f"        for (int {o2} = 0; {o2} < {n2}; ++{o2}) {{", "            R t = R(0);", PR,
              f"            for (int {s1} = 0; {s1} < {m1}; ++{s1})", PR,
              f"                for (int {s2} = 0; {s2} < {m2}; ++{s2}) t += {I} * {dref[Dn](s1, s2)};",
              f"            jk_add(c.K, (size_t)({f1} + {o1}) * c.n + {f2} + {o2}, s * t, false);", "        }"]
    L.append("}")
    return "\n".join(L) + "\n"


def main(outdir):
    os.makedirs(outdir, exist_ok=True)
    infos = []
    for cls in QUARTET_CLASSES:
        body, info = emit_class(cls)
        if team_capable(info) or info["mode"] == "program":
            body += "\n" + emit_team(cls, info)
        dig = emit_digests(cls, info)
        path = os.path.join(outdir, f"eri_class_{info['tag']}.cuh")
        text = ("// Generated by gen_eri.py: do not edit.\n#pragma once\n#include \"eri_common.cuh\"\n\n"
                + body + "\n" + dig)
        old = open(path).read() if os.path.exists(path) else None
        if old != text:
            with open(path, "w") as fh:
                fh.write(text)
        infos.append(info)
    # one translation unit per class: kernels + launcher
    for cls, info in zip(QUARTET_CLASSES, infos):
        (la, lb), (lc, ld) = cls
        t = info["tag"]
        na, nb, nc, nd = ncart(la), ncart(lb), ncart(lc), ncart(ld)
        diag = (la, lb) == (lc, ld)
        u = ["// Generated by gen_eri.py: do not edit.", f'#include "eri_class_{t}.cuh"', '#include "eri_launch.h"', "",
             f"MESS_DEFINE_CLASS_KERNELS({t}, {na}, {nb}, {nc}, {nd})"]
        team = team_capable(info) or info["mode"] == "program"
        if team:
            u.append(f"MESS_DEFINE_TEAM_KERNEL({t})")
        if diag:
            u.append(f"MESS_DEFINE_SCHWARZ_KERNEL({t}, {na}, {nb})")
        u += ["", f"cudaError_t mess_launch_{t}(const ClassLaunchArgs& a)", "{",
              "    const int T = MESS_THREADS;",
              "    if (a.kind == MESS_KIND_SCHWARZ) {",
              ]
        if diag:
            u += ["        if (a.npairs <= 0) return cudaSuccess;",
                  f"        k_schwarz_{t}<<<(a.npairs + T - 1) / T, T, 0, a.stream>>>(a.pairs, a.npairs, *a.P64_ptr, a.out);",
                  "        return cudaGetLastError();"]
        else:
            u += ["        return cudaErrorInvalidValue;"]
        u += ["    }",
              "    if (a.bin.total <= 0) return cudaSuccess;",
              "    const long long nblk = (a.bin.total + T - 1) / T;",
              "    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;",
              "    const dim3 g((unsigned)nblk);",
              "    if (a.kind == MESS_KIND_STORE) {",
              f"        k_store_{t}<<<g, T, 0, a.stream>>>(a.bin, *a.P64_ptr, a.out, a.n);",
              "    } else {",
              ] + ([
              "      if (a.team) {",
              "        // team 1: a warp per quartet (MESS_TEAM_WARPS per block); 2: the block on one quartet;",
              "        // 3: the block on one quartet, its warps splitting the primitive quartets",
              "        static int cfg[12][64];   // dynamic shared memory opt-in done, per kernel and device",
              "        const int qpb = a.team >= 2 ? 1 : MESS_TEAM_WARPS;",
              "        const long long nbt = (a.bin.total + qpb - 1) / qpb;",
              "        if (nbt > 0x7fffffffLL) return cudaErrorInvalidConfiguration;",
              "        const dim3 gt((unsigned)nbt);",
              "        if (a.team == 3) {",
              "            if (a.mode == MESS_MODE_FP64)",
              f"                return mess_team_launch<double, 0>(k_jk_team_{t}<double, 0, 32 * MESS_TEAM_WARPS, 1>, gt, team_smem_{t}<double>(), a, *a.P64_ptr, cfg[8]);",
              "            else if (a.mode == MESS_MODE_MIXED)",
              f"                return mess_team_launch<float, 1>(k_jk_team_{t}<float, 1, 32 * MESS_TEAM_WARPS, 1>, gt, team_smem_{t}<float>(), a, *a.P32_ptr, cfg[9]);",
              "            else if (a.mode == MESS_MODE_DF32)",
              f"                return mess_team_launch<df32, 3>(k_jk_team_{t}<df32, 3, 32 * MESS_TEAM_WARPS, 1>, gt, team_smem_{t}<df32>(), a, *a.Pdf_ptr, cfg[11]);",
              "            else",
              f"                return mess_team_launch<float, 2>(k_jk_team_{t}<float, 2, 32 * MESS_TEAM_WARPS, 1>, gt, team_smem_{t}<float>(), a, *a.P32_ptr, cfg[10]);",
              "        }",
              "        if (a.team == 2) {",
              "            if (a.mode == MESS_MODE_FP64)",
              f"                return mess_team_launch<double, 0>(k_jk_team_{t}<double, 0, 32 * MESS_TEAM_WARPS, 0>, gt, team_smem_{t}<double>() / MESS_TEAM_WARPS, a, *a.P64_ptr, cfg[4]);",
              "            else if (a.mode == MESS_MODE_MIXED)",
              f"                return mess_team_launch<float, 1>(k_jk_team_{t}<float, 1, 32 * MESS_TEAM_WARPS, 0>, gt, team_smem_{t}<float>() / MESS_TEAM_WARPS, a, *a.P32_ptr, cfg[5]);",
              "            else if (a.mode == MESS_MODE_DF32)",
              f"                return mess_team_launch<df32, 3>(k_jk_team_{t}<df32, 3, 32 * MESS_TEAM_WARPS, 0>, gt, team_smem_{t}<df32>() / MESS_TEAM_WARPS, a, *a.Pdf_ptr, cfg[7]);",
              "            else",
              f"                return mess_team_launch<float, 2>(k_jk_team_{t}<float, 2, 32 * MESS_TEAM_WARPS, 0>, gt, team_smem_{t}<float>() / MESS_TEAM_WARPS, a, *a.P32_ptr, cfg[6]);",
              "        }",
              "        if (a.mode == MESS_MODE_FP64)",
              f"            return mess_team_launch<double, 0>(k_jk_team_{t}<double, 0, 32, 0>, gt, team_smem_{t}<double>(), a, *a.P64_ptr, cfg[0]);",
              "        else if (a.mode == MESS_MODE_MIXED)",
              f"            return mess_team_launch<float, 1>(k_jk_team_{t}<float, 1, 32, 0>, gt, team_smem_{t}<float>(), a, *a.P32_ptr, cfg[1]);",
              "        else if (a.mode == MESS_MODE_DF32)",
              f"            return mess_team_launch<df32, 3>(k_jk_team_{t}<df32, 3, 32, 0>, gt, team_smem_{t}<df32>(), a, *a.Pdf_ptr, cfg[3]);",
              "        else",
              f"            return mess_team_launch<float, 2>(k_jk_team_{t}<float, 2, 32, 0>, gt, team_smem_{t}<float>(), a, *a.P32_ptr, cfg[2]);",
              "      }",
              ] if (team_capable(info) or info["mode"] == "program") else []) + ([
              ] + sum([[
              f"        if (a.G == {GG}) {{",
              f"            const long long nbg = (a.bin.total * {GG} + T - 1) / T;",
              "            if (nbg > 0x7fffffffLL) return cudaErrorInvalidConfiguration;",
              "            const dim3 gg((unsigned)nbg);",
              "            if (a.mode == MESS_MODE_FP64)",
              f"                k_jk_{t}<double, 0, {GG}><<<gg, T, 0, a.stream>>>(a.bin, *a.P64_ptr, dmat<double>(a), a.J, a.K, a.n);",
              "            else if (a.mode == MESS_MODE_MIXED)",
              f"                k_jk_{t}<float, 1, {GG}><<<gg, T, 0, a.stream>>>(a.bin, *a.P32_ptr, dmat<float>(a), a.J, a.K, a.n);",
              "            else if (a.mode == MESS_MODE_DF32)",
              f"                k_jk_{t}<df32, 3, {GG}><<<gg, T, 0, a.stream>>>(a.bin, *a.Pdf_ptr, dmat<df32>(a), a.J, a.K, a.n);",
              "            else",
              f"                k_jk_{t}<float, 2, {GG}><<<gg, T, 0, a.stream>>>(a.bin, *a.P32_ptr, dmat<float>(a), a.J, a.K, a.n);",
              "            return cudaGetLastError();",
              "        }"] for GG in (4, 8, 32)], []) if info["mode"] == "straight" else []) + [
              "        if (a.mode == MESS_MODE_FP64)",
              f"            k_jk_{t}<double, 0, 1><<<g, T, 0, a.stream>>>(a.bin, *a.P64_ptr, dmat<double>(a), a.J, a.K, a.n);",
              "        else if (a.mode == MESS_MODE_MIXED)",
              f"            k_jk_{t}<float, 1, 1><<<g, T, 0, a.stream>>>(a.bin, *a.P32_ptr, dmat<float>(a), a.J, a.K, a.n);",
              "        else if (a.mode == MESS_MODE_DF32)",
              f"            k_jk_{t}<df32, 3, 1><<<g, T, 0, a.stream>>>(a.bin, *a.Pdf_ptr, dmat<df32>(a), a.J, a.K, a.n);",
              "        else",
              f"            k_jk_{t}<float, 2, 1><<<g, T, 0, a.stream>>>(a.bin, *a.P32_ptr, dmat<float>(a), a.J, a.K, a.n);",
              "    }",
              "    return cudaGetLastError();",
              "}"]
        text = "\n".join(u) + "\n"
        path = os.path.join(outdir, f"eri_class_{t}.cu")
        old = open(path).read() if os.path.exists(path) else None
        if old != text:
            with open(path, "w") as fh:
                fh.write(text)
    # dispatch table
    d = ["// Generated by gen_eri.py: do not edit.", '#include "eri_launch.h"', ""]
    for info in infos:
        d.append(f"cudaError_t mess_launch_{info['tag']}(const ClassLaunchArgs& a);")
    d += ["", "const mess_class_launcher MESS_CLASS_LAUNCHERS[MESS_NUM_QCLASS] = {"]
    for info in infos:
        d.append(f"    mess_launch_{info['tag']},")
    d.append("};")
    text = "\n".join(d) + "\n"
    path = os.path.join(outdir, "eri_dispatch.cu")
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as fh:
            fh.write(text)
    # class table (host + device readable)
    tab = ["// Generated by gen_eri.py: do not edit.", "#pragma once", "",
           f"#define MESS_NUM_QCLASS {len(QUARTET_CLASSES)}", "",
           "// straight: straight-line kernels with G = 1, 4, 8 lanes per quartet (else one op-program",
           "// kernel, G = 1); team: a warp-per-quartet kernel exists",
           "typedef struct { int la, lb, lc, ld, L, nint, nacc, nvrr; long vrr_flops, hrr_flops; int straight, team; }",
           "    mess_qclass_info;",
           "static const mess_qclass_info MESS_QCLASS[MESS_NUM_QCLASS] = {"]
    for f in infos:
        st = 1 if f["mode"] == "straight" else 0
        tm = 1 if (team_capable(f) or f["mode"] == "program") else 0
        tab.append(f"    {{{f['la']}, {f['lb']}, {f['lc']}, {f['ld']}, {f['L']}, {f['nint']}, {f['nacc']}, "
                   f"{f['nvrr']}, {f['vrr_flops']}, {f['hrr_flops']}, {st}, {tm}}},")
    tab.append("};")
    text = "\n".join(tab) + "\n"
    path = os.path.join(outdir, "eri_classes.h")
    old = open(path).read() if os.path.exists(path) else None
    if old != text:
        with open(path, "w") as fh:
            fh.write(text)
    return infos


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "_gen")
