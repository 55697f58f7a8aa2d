"""The recursion programs the kernel generator emits, checked on the CPU against the oracle.

For every shell-quartet class, the Obara-Saika VRR + Head-Gordon-Pople HRR op programs (the
one-thread-per-quartet form and the level-scheduled form of the warp/block-per-quartet kernels)
are interpreted exactly as the kernels decode them, on one primitive quartet with random
exponents and centres and unit coefficients, and the resulting raw integrals are compared with
the oracle's (a different exact route, McMurchie-Davidson) for the same raw primitives.  The
level-scheduled programs are also checked for what lane-parallel execution needs: within one
level, no op reads a slot that another op of the level writes, and no two ops write one slot.
"""
import importlib.util
import math
import os

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _gen():
    path = os.path.join(ROOT, "paper_2406_03121_gb300", "csrc", "gen_eri.py")
    spec = importlib.util.spec_from_file_location("gen_eri_under_test", path)
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


GEN = _gen()
CLASSES = GEN.QUARTET_CLASSES


def _pair(a, A, b, B):
    """Gaussian product of two unit-coefficient primitives, as the pair records hold it."""
    z = a + b
    P = (a * A + b * B) / z
    K = math.sqrt(2.0) * math.pi ** 1.25 * math.exp(-a * b / z * float(np.dot(A - B, A - B))) / z
    return dict(z=z, P=P, PA=P - A, K=K, oo2z=0.5 / z, AB=A - B)


def _vrr_inputs(pb, pk, L):
    rz = 1.0 / (pb["z"] + pk["z"])
    roz, roe = pk["z"] * rz, pb["z"] * rz
    PQ = pb["P"] - pk["P"]
    T = pb["z"] * roz * float(np.dot(PQ, PQ))
    F = oracle.boys(L, T) * pb["K"] * pk["K"] * math.sqrt(rz)
    return dict(F=F, roz=roz, roe=roe, oo2ze=0.5 * rz, WP=-roz * PQ, WQ=roe * PQ)


def _vrr_op(op, Vr, Vw, H, pb, pk, x):
    """One VRR op, decoded as the kernels decode it: reads Vr, writes Vw (or accumulates into H).
    Returns (V slots read, slot written, "V" or "H")."""
    kind, t, s1, s2, s3, s4, s5, d, m1, m2 = op
    if kind == 0:
        Vw[t] = x["F"][s1]
        return [], t, "V"
    if kind == 3:
        H[s1] += Vr[t]
        return [t], s1, "H"
    if kind == 1:
        v = pb["PA"][d] * Vr[s1] + x["WP"][d] * Vr[s2]
        reads = [s1, s2]
        if m1:
            v += m1 * pb["oo2z"] * (Vr[s3] - x["roz"] * Vr[s4])
            reads += [s3, s4]
    else:
        v = pk["PA"][d] * Vr[s1] + x["WQ"][d] * Vr[s2]
        reads = [s1, s2]
        if m1:
            v += m1 * pk["oo2z"] * (Vr[s3] - x["roe"] * Vr[s4])
            reads += [s3, s4]
        if m2:
            v += m2 * x["oo2ze"] * Vr[s5]
            reads += [s5]
    Vw[t] = v
    return reads, t, "V"


def _hrr_op(op, Hr, Hw, AB, CD):
    t, s1, s2, d, side = op
    Hw[t] = Hr[s1] + (CD if side else AB)[d] * Hr[s2]
    return [s1, s2], t


def _run(prog, team, pb, pk, L):
    """Interpret a program with V and H sized exactly as the kernels declare them (a slot past the
    end raises IndexError here; on the device it would read or overwrite a neighbouring array)."""
    x = _vrr_inputs(pb, pk, L)
    nvi = max(prog["nv"], prog["nint"]) if team else prog["nv"]
    V = np.full(nvi, np.nan)
    assert prog["nh"] >= prog["nacc"]
    H = np.zeros(prog["nh"])
    H[prog["nacc"]:] = np.nan
    if team:
        # lane-parallel levels: every op of a level sees the values from before the level
        lv = prog["vlev"]
        for k in range(len(lv) - 1):
            Vb = V.copy()
            vreads, vwrites, hwrites = set(), [], []
            for op in prog["vrr"][lv[k]:lv[k + 1]]:
                reads, w, arr = _vrr_op(op, Vb, V, H, pb, pk, x)
                vreads.update(reads)
                (vwrites if arr == "V" else hwrites).append(w)
            assert len(set(vwrites)) == len(vwrites), "two VRR ops of one level write the same slot"
            assert len(set(hwrites)) == len(hwrites), "two accumulations of one level hit the same slot"
            assert not (vreads & set(vwrites)), "an op reads a slot written in its own level"
        hl = prog["hlev"]
        for k in range(len(hl) - 1):
            Hb = H.copy()
            reads_all, writes = set(), []
            for op in prog["hrr"][hl[k]:hl[k + 1]]:
                reads, w = _hrr_op(op, Hb, H, pb["AB"], pk["AB"])
                writes.append(w)
                reads_all.update(reads)
            assert len(set(writes)) == len(writes), "two HRR ops of one level write the same slot"
            assert not (reads_all & set(writes)), "an HRR op reads a slot written in its own level"
    else:
        for op in prog["vrr"]:
            _vrr_op(op, V, V, H, pb, pk, x)
        for op in prog["hrr"]:
            _hrr_op(op, H, H, pb["AB"], pk["AB"])
    out = np.array([H[s] for s, _ in prog["fin"]])
    assert np.all(np.isfinite(out)), "a final integral reads a slot never written"
    if team:
        # the warp/block kernels store the final integrals over the V region before the digestion
        for k, (s, _) in enumerate(prog["fin"]):
            V[k] = H[s]
        assert np.array_equal(V[:len(out)], out)
    return out


def _oracle_raw(cls, exps, centres):
    """Raw-primitive integrals (unit coefficients, no normalisation) in the kernels' index order."""
    (la, lb), (lc, ld) = cls
    ls = [la, lb, lc, ld]
    center, lmn, first = [], [], []
    for l, R in zip(ls, centres):
        first.append(len(lmn))
        for comp in GEN.cart(l):
            center.append(R)
            lmn.append(comp)
    n = len(lmn)
    nprim = np.ones(n, dtype=np.int32)
    poff = np.arange(n, dtype=np.int32)
    ex = np.array([exps[s] for s in range(4) for _ in GEN.cart(ls[s])], dtype=np.float64)
    b = oracle.Basis(n, np.ascontiguousarray(np.array(center, dtype=np.float64)),
                     np.ascontiguousarray(np.array(lmn, dtype=np.int32)), nprim, poff, ex,
                     np.ones(n), np.arange(n, dtype=np.int32), n, np.zeros(n, dtype=np.int32),
                     np.zeros(1, dtype=np.int32), np.zeros((1, 3)))
    out = []
    for i in range(GEN.ncart(la)):
        for j in range(GEN.ncart(lb)):
            for k in range(GEN.ncart(lc)):
                for m in range(GEN.ncart(ld)):
                    out.append(oracle.eri(b, first[0] + i, first[1] + j, first[2] + k, first[3] + m))
    return np.array(out)


@pytest.mark.parametrize("cls", CLASSES, ids=[GEN.tag(c) for c in CLASSES])
def test_programs_match_oracle(cls):
    (la, lb), (lc, ld) = cls
    rng = np.random.default_rng(100 + 7 * la + 5 * lb + 3 * lc + ld)
    L = la + lb + lc + ld
    for trial in range(2):
        exps = rng.uniform(0.3, 2.5, 4)
        centres = [rng.normal(scale=0.8, size=3) for _ in range(4)]
        if trial == 1:
            centres[1] = centres[0].copy()        # one-centre bra pair (AB = 0)
        pb = _pair(exps[0], centres[0], exps[1], centres[1])
        pk = _pair(exps[2], centres[2], exps[3], centres[3])
        ref = _oracle_raw(cls, exps, centres)
        scale = np.abs(ref).max()
        team = GEN.build_team_program(cls)
        got = _run(team, True, pb, pk, L)
        assert np.abs(got - ref).max() <= 1e-11 * scale + 1e-14, "level-scheduled program"
        prog = GEN.build_program(cls)
        got = _run(prog, False, pb, pk, L)
        assert np.abs(got - ref).max() <= 1e-11 * scale + 1e-14, "op program"


@pytest.mark.parametrize("cls", CLASSES, ids=[GEN.tag(c) for c in CLASSES])
def test_component_scales(cls):
    """The per-integral scale of the final values is the product of the four components' factors
    sqrt((2L-1)!! / ((2l-1)!! (2m-1)!! (2n-1)!!)), which turns the x^L-normalised shell into unit
    norm for every component (1 for s and p, sqrt(3) off-diagonal for d: xy, xz, yz)."""
    (la, lb), (lc, ld) = cls
    prog = GEN.build_team_program(cls)
    d = {(2, 0, 0): 1.0, (0, 2, 0): 1.0, (0, 0, 2): 1.0, (1, 1, 0): math.sqrt(3.0), (1, 0, 1): math.sqrt(3.0),
         (0, 1, 1): math.sqrt(3.0)}
    fac = lambda l, c: d[c] if l == 2 else 1.0  # noqa: E731
    k = 0
    for a in GEN.cart(la):
        for b in GEN.cart(lb):
            for c in GEN.cart(lc):
                for e in GEN.cart(ld):
                    want = fac(la, a) * fac(lb, b) * fac(lc, c) * fac(ld, e)
                    assert prog["fin"][k][1] == pytest.approx(want, rel=1e-15)
                    k += 1


def _decode_vrr(w):
    """One uint4 VRR word decoded as the kernels decode it."""
    x, y, z, ww = w
    return dict(kind=x & 3, d=(x >> 2) & 3, m1=(x >> 4) & 15, m2=(x >> 8) & 15, t=x >> 16,
                s1=y & 0xFFFF, s2=y >> 16, s3=z & 0xFFFF, s4=z >> 16, s5=ww)


@pytest.mark.parametrize("cls", CLASSES, ids=[GEN.tag(c) for c in CLASSES])
def test_program_slots_in_bounds(cls):
    """Every slot index a program names is below the size of the array the kernel declares for it
    (V: NV, or max(NV, NINT) in the warp/block kernels, which store the integrals over V; H: NH, whose
    first NACC slots hold the contracted values), and the packed words the generator emits decode
    back to the same fields."""
    (la, lb), (lc, ld) = cls
    L = la + lb + lc + ld
    for prog, nvi in ((GEN.build_program(cls), None), (GEN.build_team_program(cls), "team")):
        nv = max(prog["nv"], prog["nint"]) if nvi else prog["nv"]
        nh, nacc = prog["nh"], prog["nacc"]
        assert nacc <= nh
        for op in prog["vrr"]:
            kind, t, s1, s2, s3, s4, s5, d, m1, m2 = op
            word = (kind | (d << 2) | (m1 << 4) | (m2 << 8) | (t << 16), s1 | (s2 << 16), s3 | (s4 << 16), s5)
            assert all(0 <= w < 2 ** 32 for w in word)
            dec = _decode_vrr(word)
            assert (dec["kind"], dec["t"], dec["d"], dec["m1"], dec["m2"]) == (kind, t, d, m1, m2)
            assert dec["t"] < prog["nv"]
            if kind == 0:
                assert dec["s1"] <= L                       # F[m], m <= L
            elif kind == 3:
                assert dec["s1"] < nacc                     # H[acc] += V[t]
            else:
                assert max(dec["s1"], dec["s2"]) < prog["nv"]
                if m1:
                    assert max(dec["s3"], dec["s4"]) < prog["nv"]
                if m2:
                    assert dec["s5"] < prog["nv"]
        for (t, s1, s2, d, side) in prog["hrr"]:
            wx, wy = t | (d << 16) | (side << 18), s1 | (s2 << 16)
            assert (wx & 0xFFFF, (wx >> 16) & 3, (wx >> 18) & 1, wy & 0xFFFF, wy >> 16) == (t, d, side, s1, s2)
            assert max(t, s1, s2) < nh
        assert all(f < nh for f, _ in prog["fin"])
        assert len(prog["fin"]) <= nv or not nvi


@pytest.mark.parametrize("cls", CLASSES, ids=[GEN.tag(c) for c in CLASSES])
def test_programs_read_only_written_slots(cls):
    """In program order (one thread per quartet) and level by level (warp/block kernels), every slot
    an op reads holds a value written earlier - H's first NACC slots hold the contracted values from
    the start - so no kernel reads an indeterminate local or shared value (undefined behaviour that a
    compiler may exploit)."""
    for prog, team in ((GEN.build_program(cls), False), (GEN.build_team_program(cls), True)):
        vw, hw = set(), set(range(prog["nacc"]))
        def vrr(op):
            kind, t, s1, s2, s3, s4, s5, d, m1, m2 = op
            if kind == 0:
                return [], ("V", t)
            if kind == 3:
                return [("V", t)], ("H", s1)
            reads = [s1, s2] + ([s3, s4] if m1 else []) + ([s5] if (kind == 2 and m2) else [])
            return [("V", x) for x in reads], ("V", t)
        groups = ([prog["vrr"][a:b] for a, b in zip(prog["vlev"][:-1], prog["vlev"][1:])] if team
                  else [[op] for op in prog["vrr"]])
        for ops in groups:
            writes = []
            for op in ops:
                reads, w = vrr(op)
                for arr, x in reads:
                    assert x in (vw if arr == "V" else hw), (GEN.tag(cls), "VRR reads", arr, x)
                writes.append(w)
            for arr, x in writes:
                (vw if arr == "V" else hw).add(x)
        hgroups = ([prog["hrr"][a:b] for a, b in zip(prog["hlev"][:-1], prog["hlev"][1:])] if team
                   else [[op] for op in prog["hrr"]])
        for ops in hgroups:
            for (t, s1, s2, d, side) in ops:
                assert s1 in hw and s2 in hw, (GEN.tag(cls), "HRR reads", s1, s2)
            for (t, s1, s2, d, side) in ops:
                hw.add(t)
        assert all(f in hw for f, _ in prog["fin"])


@pytest.mark.parametrize("cls", CLASSES, ids=[GEN.tag(c) for c in CLASSES])
def test_interpreter_kernels_stage_no_density(cls):
    """Where a one-thread kernel runs the op-program interpreter (the op-program classes, and the
    double-float path of the larger straight-line classes), its digestion reads the density through
    the read-only cache and never stages it in arrays: a one-thread kernel that inlined the
    interpreter and also staged the density blocks in local arrays was built with a stack frame
    smaller than its live arrays, and its integrals came out as density values (the same source with
    the interpreter not inlined was exact).  The straight-line code stages the blocks in registers."""
    t = GEN.tag(cls)
    body, info = GEN.emit_class(cls)
    text = GEN.emit_digests(cls, info)
    staged = lambda txt: any(f"R {nm}[" in txt for nm in ("Dab", "Dcd", "Dac", "Dad", "Dbc", "Dbd"))
    if info["mode"] == "program":
        assert not staged(text)
    elif GEN.df32_program(info):
        assert f"eri_program<" in body and "std::is_same<R, df32>::value && G == 1" in body
        ro = GEN.emit_digest(cls, unroll=False, name=f"digest_{t}_ro")
        assert ro in text and not staged(ro)
        assert f"if constexpr (std::is_same<R, df32>::value) digest_{t}_ro<R>(I, c, s);" in text
    else:
        assert "eri_program<" not in body and staged(text)
    src = open(os.path.join(ROOT, "paper_2406_03121_gb300", "csrc", "gen_eri.py")).read()
    assert "dig = emit_digests(cls, info)" in src


def _lane_split_visits(nb, nk, G, g, guard=True):
    """The lane-split primitive loop of the straight-line kernels (G lanes, lane g), index logic only:
    returns the (bra, ket) primitive indices lane g visits, or None if it runs past a step limit."""
    b0, k0 = 0, 0
    k1 = k0 + nk
    b1 = b0 + (nb if nk > 0 else 0)
    ib, ik, visits, steps = b0, k0 + g, [], 0
    while ik >= k1 and (ib < b1 or not guard):
        ik -= nk; ib += 1; steps += 1
        if steps > 10000:
            return None
    while ib < b1:
        visits.append((ib, ik))
        ik += G
        while ik >= k1 and (ib < b1 or not guard):
            ik -= nk; ib += 1; steps += 1
            if steps > 10000:
                return None
    return visits


@pytest.mark.parametrize("G", [4, 8, 32])
def test_lane_split_loop_terminates_and_covers(G):
    """The lanes of a group visit every primitive quartet exactly once and always leave the loop, also
    for a ket pair without primitives (nk = 0), where the unguarded index normalisation never ends."""
    for nb in range(0, 5):
        for nk in range(0, 7):
            seen = []
            for g in range(G):
                v = _lane_split_visits(nb, nk, G, g)
                assert v is not None, (nb, nk, G, g)
                seen += v
            assert sorted(seen) == [(b, k) for b in range(nb if nk else 0) for k in range(nk)]
    assert _lane_split_visits(3, 0, G, 1, guard=False) is None     # what the guard prevents
    _, info = GEN.emit_class(((1, 0), (1, 0)))
    body, _ = GEN.emit_class_straight(((1, 0), (1, 0)))
    assert body.count("while (ik >= k1 && ib < b1) { ik -= nk; ++ib; }") == 2
    assert "b1 = b0 + ((live && nk > 0) ? P.pp_n[bp] : 0);" in body
