"""CPU check of the generated VRR node tables of the warp-cooperative
kernel (classes with la+lb+lc+ld >= 5).

The tables (paper_1303_4916_gb300/csrc/gen_eri.py) encode the vertical
recurrence of the Obara-Saika scheme, in Head-Gordon-Pople form, as nodes
out = c0 x0 + c1 x1 [+ c2 (x2 - c3 x3)] [+ c4 x4] over shared-memory slots,
grouped in dependency levels.  Here the tables are decoded and evaluated
exactly as the kernel does, for random values of the per-primitive-quartet
quantities, and every target [e0|f0]^(0) is compared with a memoised
recursion written out in this file from the textbook relations:

  [e+1_i | f]^(m) = PA_i [e|f]^(m) + WP_i [e|f]^(m+1)
                    + e_i/(2p) ([e-1_i|f]^(m) - (rho/p) [e-1_i|f]^(m+1))
                    + f_i/(2(p+q)) [e|f-1_i]^(m+1)
  [e | f+1_i]^(m) = QC_i [e|f]^(m) + WQ_i [e|f]^(m+1)
                    + f_i/(2q) ([e|f-1_i]^(m) - (rho/q) [e|f-1_i]^(m+1))
                    + e_i/(2(p+q)) [e-1_i|f]^(m+1)

with [0|0]^(m) = B_m.  The recursion here always lowers e first (the
generator lowers f first), so the two follow different paths through the
same relations.
"""
import importlib.util
import os
import random
from functools import lru_cache

import pytest

GEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1303_4916_gb300", "csrc", "gen_eri.py")


@pytest.fixture(scope="module")
def gen():
    spec = importlib.util.spec_from_file_location("gen_eri", GEN)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _reference(q, B):
    """[e|f]^(m) by the relations above, lowering e before f."""
    @lru_cache(maxsize=None)
    def val(e, f, m):
        if sum(e) == 0 and sum(f) == 0:
            return B[m]
        if sum(e) > 0:
            i = next(k for k in range(3) if e[k] > 0)
            e1 = tuple(x - (k == i) for k, x in enumerate(e))
            r = q["PA"][i] * val(e1, f, m) + q["WP"][i] * val(e1, f, m + 1)
            if e1[i] > 0:
                e2 = tuple(x - (k == i) for k, x in enumerate(e1))
                r += e1[i] * q["o2p"] * (val(e2, f, m) - q["rp"] * val(e2, f, m + 1))
            if f[i] > 0:
                f1 = tuple(x - (k == i) for k, x in enumerate(f))
                r += f[i] * q["o2pq"] * val(e1, f1, m + 1)
            return r
        i = next(k for k in range(3) if f[k] > 0)
        f1 = tuple(x - (k == i) for k, x in enumerate(f))
        r = q["QC"][i] * val(e, f1, m) + q["WQ"][i] * val(e, f1, m + 1)
        if f1[i] > 0:
            f2 = tuple(x - (k == i) for k, x in enumerate(f1))
            r += f1[i] * q["o2q"] * (val(e, f2, m) - q["rq"] * val(e, f2, m + 1))
        return r
    return val


def _coefficients(gen, q):
    """The kernel's coefficient vector for the values q, by name."""
    cv = {"zero": 0.0, "rp": q["rp"], "rq": q["rq"]}
    for i in range(3):
        for n in ("PA", "WP", "QC", "WQ"):
            cv[f"{n}{i}"] = q[n][i]
    for k in range(1, 9):
        cv[f"o2p{k}"] = k * q["o2p"]
        cv[f"o2q{k}"] = k * q["o2q"]
        cv[f"o2pq{k}"] = k * q["o2pq"]
    return [cv[n] for n in gen.COEF_NAMES]


def _evaluate_tables(nslot, bounds, words, tgt, cv, B):
    """Level by level, each level's nodes reading only earlier slots."""
    s = [None] * nslot
    for m, b in enumerate(B):
        s[m] = b
    lo = 0
    for hi in bounds:
        level_out = {}
        for w0, w1, w2, w3 in words[lo:hi]:
            x = [w0 >> 16, w1 & 0xFFFF, w1 >> 16, w2 & 0xFFFF, w2 >> 16]
            c = [(w3 >> (6 * k)) & 63 for k in range(5)]
            v = cv[c[0]] * s[x[0]] + cv[c[1]] * s[x[1]]
            if w3 & (1 << 30):
                v += cv[c[2]] * (s[x[2]] - cv[c[3]] * s[x[3]])
            else:
                assert c[2] == 0
            if w3 & (1 << 31):
                v += cv[c[4]] * s[x[4]]
            else:
                assert c[4] == 0
            level_out[w0 & 0xFFFF] = v
        for k, v in level_out.items():   # written after the level: no same-level reads
            assert s[k] is None
            s[k] = v
        lo = hi
    return [s[t] for t in tgt]


def test_cooperative_tables_match_the_recurrence(gen):
    rng = random.Random(2024)
    _, classes = gen.classes(2)
    heavy = [c for c in classes if sum(c) >= gen.COOP_LMIN]
    assert len(heavy) == 8
    for cls in heavy:
        v = gen.VRR(*cls)
        v.build()
        nslot, bounds, words, tgt = gen.coop_schedule(v)
        for trial in range(3):
            q = {n: [rng.uniform(-1.0, 1.0) for _ in range(3)] for n in ("PA", "WP", "QC", "WQ")}
            q.update(rp=rng.uniform(0.1, 0.9), rq=rng.uniform(0.1, 0.9), o2p=rng.uniform(0.05, 2.0),
                     o2q=rng.uniform(0.05, 2.0), o2pq=rng.uniform(0.05, 1.0))
            B = [rng.uniform(0.1, 1.0) for _ in range(v.L + 1)]
            got = _evaluate_tables(nslot, bounds, words, tgt, _coefficients(gen, q), B)
            ref = _reference(q, tuple(B))
            expect = [ref(e, f, 0) for e in v.E.comps for f in v.F.comps]
            scale = max(1.0, max(abs(x) for x in expect))
            err = max(abs(a - b) for a, b in zip(got, expect)) / scale
            assert err < 1e-12, (cls, trial, err)
