#!/usr/bin/env python3
"""Generate the per-class recurrence code for the ERI kernels.

For every canonical shell-quartet class (la lb | lc ld) with la >= lb,
lc >= ld and pair class (la,lb) >= (lc,ld), emit a struct with

* ``vrr``: the Obara-Saika vertical recurrence, in the Head-Gordon-Pople
  arrangement, from [00|00]^(m) = B_m (prefactor times the Boys function
  F_m(T)) to the primitive integrals [e0|f0]^(0) for la <= |e| <= la+lb,
  lc <= |f| <= lc+ld, which it adds into the contracted accumulators;

      [e+1_i,0|00]^(m) = PA_i [e0|00]^(m) + WP_i [e0|00]^(m+1)
                         + e_i/(2 zeta) ([e-1_i,0|00]^(m) - rho/zeta [e-1_i,0|00]^(m+1))
      [e0|f+1_i,0]^(m) = QC_i [e0|f0]^(m) + WQ_i [e0|f0]^(m+1)
                         + f_i/(2 eta) ([e0|f-1_i,0]^(m) - rho/eta [e0|f-1_i,0]^(m+1))
                         + e_i/(2(zeta+eta)) [e-1_i,0|f0]^(m+1)

* ``hrr``: the horizontal recurrence on the contracted integrals, first on
  the bra then on the ket,

      (a, b+1_i| = (a+1_i, b| + AB_i (a, b|     (AB = A - B)
      |c, d+1_i) = |c+1_i, d) + CD_i |c, d)     (CD = C - D)

  writing the Cartesian block out[((a*NB + b)*NC + c)*ND + d].

The recurrences are the closed-form relations between Gaussian integrals
(Obara & Saika 1986; Head-Gordon & Pople 1988) that the paper's ERI, Eq. 5,
admits; the paper itself evaluates them by Rys quadrature.  Exact operation
counts are written next to each class for the roofline accounting.

Usage: gen_eri.py OUT_HEADER [LMAX]
"""
from __future__ import annotations

import sys


def cart(l):
    out = []
    for x in range(l, -1, -1):
        for y in range(l - x, -1, -1):
            out.append((x, y, l - x - y))
    return out


def ncart(l):
    return (l + 1) * (l + 2) // 2


def tl(v):
    return sum(v)


def add(v, i, k):
    w = list(v)
    w[i] += k
    return tuple(w)


def coef(k, name):
    """k * name as a source expression (k = 1 needs no multiplication)."""
    return name if k == 1 else f"((R){k} * {name})"


def render(terms, init=None):
    """Source of init + sum of terms as nested fused multiply-adds
    fmac(a, b, c) = a*b + c (one FMA in FP64/FP32, one fused double-float
    step in df64): c0*x0, then fmac(c1, x1, .), and c*(x2 - c3*x3) as
    fmac(c, fmac(-c3, x3, x2), .)."""
    def one(t, acc):
        if t[0] == "p":
            return f"{t[1]} * {t[2]}" if acc is None else f"fmac({t[1]}, {t[2]}, {acc})"
        inner = f"fmac(-{t[3]}, {t[4]}, {t[2]})"
        return f"{t[1]} * {inner}" if acc is None else f"fmac({t[1]}, {inner}, {acc})"
    expr = init
    for t in terms:
        expr = one(t, expr)
    return expr


def pick_axis(v):
    # the axis with the largest power; ties broken towards x
    best = 0
    for i in range(3):
        if v[i] > v[best]:
            best = i
    return best


class Range:
    """Cartesian components of all l in [lo, hi], concatenated."""

    def __init__(self, lo, hi):
        self.lo, self.hi = lo, hi
        self.comps = []
        for l in range(lo, hi + 1):
            self.comps.extend(cart(l))
        self.index = {c: k for k, c in enumerate(self.comps)}

    def __len__(self):
        return len(self.comps)


class VRR:
    def __init__(self, la, lb, lc, ld):
        self.L = la + lb + lc + ld
        self.E = Range(la, la + lb)
        self.F = Range(lc, lc + ld)
        self.memo = {}
        self.lines = []
        self.nvar = 0
        self.flops = 0
        self.nodes = []   # (name, key, node spec) in dependency order
        self.exprs = {}   # name -> right-hand side

    def get(self, e, f, m):
        key = (e, f, m)
        if key in self.memo:
            return self.memo[key]
        if tl(e) == 0 and tl(f) == 0:
            name = f"B[{m}]"
            self.memo[key] = name
            return name
        # terms: ("p", c, x) is c*x; ("d", c, x2, c3, x3) is c*(x2 - c3*x3)
        terms = []
        # node spec: value = c0*x0 + c1*x1 + c2*(x2 - c3*x3) + c4*x4, inputs as
        # DAG keys (None = absent), coefficients as names in the coefficient vector
        node = {"x": [None] * 5, "c": ["zero"] * 5}
        if tl(f) > 0:
            i = pick_axis(f)
            f1 = add(f, i, -1)
            terms.append(("p", f"QC[{i}]", self.get(e, f1, m)))
            terms.append(("p", f"WQ[{i}]", self.get(e, f1, m + 1)))
            node["x"][0], node["c"][0] = (e, f1, m), f"QC{i}"
            node["x"][1], node["c"][1] = (e, f1, m + 1), f"WQ{i}"
            nflop = 3
            if f1[i] > 0:
                f2 = add(f1, i, -1)
                terms.append(("d", coef(f1[i], "o2q"), self.get(e, f2, m), "rq", self.get(e, f2, m + 1)))
                node["x"][2], node["x"][3] = (e, f2, m), (e, f2, m + 1)
                node["c"][2], node["c"][3] = f"o2q{f1[i]}", "rq"
                nflop += 4 if f1[i] > 1 else 3
            if e[i] > 0:
                e1 = add(e, i, -1)
                terms.append(("p", coef(e[i], "o2pq"), self.get(e1, f1, m + 1)))
                node["x"][4], node["c"][4] = (e1, f1, m + 1), f"o2pq{e[i]}"
                nflop += 3 if e[i] > 1 else 2
        else:
            i = pick_axis(e)
            e1 = add(e, i, -1)
            terms.append(("p", f"PA[{i}]", self.get(e1, f, m)))
            terms.append(("p", f"WP[{i}]", self.get(e1, f, m + 1)))
            node["x"][0], node["c"][0] = (e1, f, m), f"PA{i}"
            node["x"][1], node["c"][1] = (e1, f, m + 1), f"WP{i}"
            nflop = 3
            if e1[i] > 0:
                e2 = add(e1, i, -1)
                terms.append(("d", coef(e1[i], "o2p"), self.get(e2, f, m), "rp", self.get(e2, f, m + 1)))
                node["x"][2], node["x"][3] = (e2, f, m), (e2, f, m + 1)
                node["c"][2], node["c"][3] = f"o2p{e1[i]}", "rp"
                nflop += 4 if e1[i] > 1 else 3
        name = f"v{self.nvar}"
        self.nvar += 1
        self.lines.append(f"const R {name} = {render(terms)};")
        self.exprs[name] = terms
        self.flops += nflop
        self.memo[key] = name
        self.nodes.append((name, key, node))
        return name

    def build(self):
        targets = []
        for fi, f in enumerate(self.F.comps):
            for ei, e in enumerate(self.E.comps):
                targets.append((ei * len(self.F) + fi, self.get(e, f, 0)))
        # a target no other node reads is folded into its accumulation:
        # acc = fmac(c1, x1, fmac(c0, x0, acc)), one fused step per term
        used = set()
        for name, key, node in self.nodes:
            for x in node["x"]:
                if x is not None:
                    used.add(self.memo[x])
        folded = {v for _, v in targets if v in self.exprs and v not in used}
        lines = [ln for ln in self.lines if ln.split(" = ")[0].split()[-1] not in folded]
        acc_lines = []
        for k, v in targets:
            if v in folded:
                acc_lines.append(f"acc[{k}] = {render(self.exprs[v], f'acc[{k}]')};")
            else:
                acc_lines.append(f"acc[{k}] += {v};")
        self.flops += len(acc_lines)
        return lines + acc_lines


class HRR:
    def __init__(self, la, lb, lc, ld):
        self.la, self.lb, self.lc, self.ld = la, lb, lc, ld
        self.E = Range(la, la + lb)
        self.F = Range(lc, lc + ld)
        self.flops = 0

    def _side(self, l1, l2, leaf, tmp_prefix, dvec):
        memo = {}
        lines = []
        cnt = [0]
        flops = [0]

        def get(a, b):
            key = (a, b)
            if key in memo:
                return memo[key]
            if tl(b) == 0:
                memo[key] = leaf(a)
                return memo[key]
            i = pick_axis(b)
            b1 = add(b, i, -1)
            x = get(add(a, i, 1), b1)
            y = get(a, b1)
            name = f"{tmp_prefix}{cnt[0]}"
            cnt[0] += 1
            lines.append(f"const R {name} = {x} + {dvec}[{i}] * {y};")
            flops[0] += 2
            memo[key] = name
            return name

        outs = []
        for a in cart(l1):
            for b in cart(l2):
                outs.append(get(a, b))
        return lines, outs, flops[0]

    def build_rows(self):
        """Per-row HRR bodies: bra for one f (in: x[e], out: y[ab]) and ket
        for one ab (in: x[f], out: y[cd])."""
        lines_b, outs_b, fb = self._side(self.la, self.lb, lambda a: f"x[{self.E.index[a]}]", "h", "AB")
        bra = lines_b + [f"y[{k}] = {o};" for k, o in enumerate(outs_b)]
        lines_k, outs_k, fk = self._side(self.lc, self.ld, lambda c: f"x[{self.F.index[c]}]", "k", "CD")
        ket = lines_k + [f"y[{k}] = {o};" for k, o in enumerate(outs_k)]
        return bra, ket

    def build(self):
        NE, NF = len(self.E), len(self.F)
        NA, NB, NC, ND = ncart(self.la), ncart(self.lb), ncart(self.lc), ncart(self.ld)
        code = []
        # bra: hb[ab * NF + f] from acc[e * NF + f]
        lines, outs, fl = self._side(self.la, self.lb, lambda a: f"acc[{self.E.index[a]} * {NF} + f]",
                                     "h", "AB")
        code.append(f"#pragma unroll")
        code.append(f"for (int f = 0; f < {NF}; ++f) {{")
        code += ["  " + s for s in lines]
        for k, o in enumerate(outs):
            code.append(f"  hb[{k} * {NF} + f] = {o};")
        code.append("}")
        self.flops += fl * NF
        # ket: out[ab * NC*ND + cd] from hb[ab * NF + f]
        lines, outs, fl = self._side(self.lc, self.ld, lambda c: f"hb[ab * {NF} + {self.F.index[c]}]",
                                     "k", "CD")
        code.append(f"#pragma unroll")
        code.append(f"for (int ab = 0; ab < {NA * NB}; ++ab) {{")
        code += ["  " + s for s in lines]
        for k, o in enumerate(outs):
            code.append(f"  out[ab * {NC * ND} + {k}] = {o};")
        code.append("}")
        self.flops += fl * NA * NB
        return code


# Coefficient vector of one primitive quartet, shared by the lanes of a
# warp in the cooperative kernels (index: name).
COEF_NAMES = (["zero"] + [f"PA{i}" for i in range(3)] + [f"WP{i}" for i in range(3)] + [f"QC{i}" for i in range(3)]
              + [f"WQ{i}" for i in range(3)] + ["rp", "rq"] + [f"o2p{k}" for k in range(1, 9)]
              + [f"o2q{k}" for k in range(1, 9)] + [f"o2pq{k}" for k in range(1, 9)])
COEF_INDEX = {n: i for i, n in enumerate(COEF_NAMES)}
COOP_LMIN = 5   # classes with la+lb+lc+ld >= this use the warp-cooperative kernel


def coop_schedule(v):
    """Slots and dependency levels of the VRR DAG of class v (built)."""
    level = {((0, 0, 0), (0, 0, 0), m): 0 for m in range(v.L + 1)}   # leaves B[m]
    recs = []
    for name, key, node in v.nodes:
        ins = [x for x in node["x"] if x is not None]
        lv = 1 + max(level[x] for x in ins)
        level[key] = lv
        recs.append((lv, key, node))

    # level order; inside a level, nodes grouped by which optional terms they
    # have (type bit 0: the c2 (x2 - c3 x3) term, bit 1: the c4 x4 term), so
    # that the 32 lanes of a warp mostly take the same branch, then by their
    # coefficient indices, so that the lanes of a round mostly read the same
    # coefficients (shared-memory broadcast instead of bank conflicts)
    def ntype(node):
        return int(node["c"][2] != "zero") | (int(node["c"][4] != "zero") << 1)
    recs.sort(key=lambda r: (r[0], ntype(r[2]), tuple(COEF_INDEX[n] for n in r[2]["c"])))
    # slots: leaves first, then the nodes in evaluation order, so that a
    # round's 32 outputs are consecutive
    slot = {((0, 0, 0), (0, 0, 0), m): m for m in range(v.L + 1)}
    for lv, key, node in recs:
        slot[key] = len(slot)
    nlev = max([r[0] for r in recs], default=0)
    bounds = [0] * (nlev + 2)
    for lv, _, _ in recs:
        bounds[lv + 1] += 1
    for k in range(1, len(bounds)):
        bounds[k] += bounds[k - 1]
    words = []
    for lv, key, node in recs:
        x = [slot[t] if t is not None else 0 for t in node["x"]]
        c = [COEF_INDEX[n] for n in node["c"]]
        assert max(x) < 65536 and max(c) < 64
        w0 = slot[key] | (x[0] << 16)
        w1 = x[1] | (x[2] << 16)
        w2 = x[3] | (x[4] << 16)
        w3 = c[0] | (c[1] << 6) | (c[2] << 12) | (c[3] << 18) | (c[4] << 24) | (ntype(node) << 30)
        words.append((w0, w1, w2, w3))
    targets = []
    for fi, f in enumerate(v.F.comps):
        for ei, e in enumerate(v.E.comps):
            targets.append(slot[(e, f, 0)] if (e, f, 0) in slot else None)
    # acc order is ei * NF + fi
    tgt = [0] * (len(v.E) * len(v.F))
    for fi, f in enumerate(v.F.comps):
        for ei, e in enumerate(v.E.comps):
            tgt[ei * len(v.F) + fi] = slot[(e, f, 0)]
    return len(slot), bounds[1:], words, tgt


LNAME = "spdfghik"


def classes(lmax):
    pairs = [(a, b) for a in range(lmax + 1) for b in range(a + 1)]   # pair classes, ordered
    out = []
    for bi, (la, lb) in enumerate(pairs):
        for ki, (lc, ld) in enumerate(pairs[: bi + 1]):
            out.append((la, lb, lc, ld))
    return pairs, out


def emit(lmax):
    pairs, cls = classes(lmax)
    o = []
    o.append("// Generated by gen_eri.py -- do not edit by hand.")
    o.append("// Obara-Saika VRR (Head-Gordon-Pople arrangement) and HRR per class.")
    o.append("#pragma once")
    o.append(f"#define HF_GEN_LMAX {lmax}")
    o.append(f"#define HF_GEN_NPAIRCLASS {len(pairs)}")
    o.append(f"#define HF_GEN_NCLASS {len(cls)}")
    o.append("")
    o.append("namespace hfgen {")
    o.append("")
    o.append("// a * b + c, fused, for the built-in arithmetic types; the double-float type")
    o.append("// brings its own fmac, found by argument-dependent lookup")
    o.append("__device__ __forceinline__ double fmac(double a, double b, double c) { return fma(a, b, c); }")
    o.append("__device__ __forceinline__ float fmac(float a, float b, float c) { return fmaf(a, b, c); }")
    o.append("")
    table = []
    coop_tables = []
    for (la, lb, lc, ld) in cls:
        v = VRR(la, lb, lc, ld)
        vlines = v.build()
        h = HRR(la, lb, lc, ld)
        hlines = h.build()
        NE, NF = len(v.E), len(v.F)
        name = f"C_{LNAME[la]}{LNAME[lb]}_{LNAME[lc]}{LNAME[ld]}"
        table.append((name, la, lb, lc, ld, v.flops, h.flops))
        o.append(f"// ({LNAME[la]}{LNAME[lb]}|{LNAME[lc]}{LNAME[ld]}): VRR {v.flops} flops per primitive "
                 f"quartet, HRR {h.flops} flops per contracted quartet")
        o.append(f"struct {name} {{")
        o.append(f"  static constexpr int LA = {la}, LB = {lb}, LC = {lc}, LD = {ld}, L = {la + lb + lc + ld};")
        o.append(f"  static constexpr int NE = {NE}, NF = {NF};")
        o.append(f"  static constexpr int NA = {ncart(la)}, NB = {ncart(lb)}, NC = {ncart(lc)}, ND = {ncart(ld)};")
        o.append(f"  static constexpr int VRR_FLOPS = {v.flops}, HRR_FLOPS = {h.flops};")
        o.append("  template <typename R>")
        o.append("  __device__ __forceinline__ static void vrr(R* __restrict__ acc, const R* __restrict__ B,")
        o.append("      const R* PA, const R* WP, const R* QC, const R* WQ,")
        o.append("      R o2p, R o2q, R o2pq, R rp, R rq) {")
        o.append("    (void)PA; (void)WP; (void)QC; (void)WQ; (void)o2p; (void)o2q; (void)o2pq; (void)rp; (void)rq;")
        o += ["    " + s for s in vlines]
        o.append("  }")
        L = la + lb + lc + ld
        coop = L >= COOP_LMIN
        o.append(f"  static constexpr bool COOP = {'true' if coop else 'false'};")
        if coop:
            nslot, bounds, words, tgt = coop_schedule(v)
            o.append(f"  static constexpr int NSLOT = {nslot}, NNODE = {len(words)}, NLEV = {len(bounds)};")
            br, kt = h.build_rows()
            o.append("  template <typename R>")
            o.append("  __device__ __forceinline__ static void hrr_bra_row(const R* __restrict__ x, R* __restrict__ y, const R* AB) {")
            o.append("    (void)AB;")
            o += ["    " + q for q in br]
            o.append("  }")
            o.append("  template <typename R>")
            o.append("  __device__ __forceinline__ static void hrr_ket_row(const R* __restrict__ x, R* __restrict__ y, const R* CD) {")
            o.append("    (void)CD;")
            o += ["    " + q for q in kt]
            o.append("  }")
            coop_tables.append((name, words, bounds, tgt))
        o.append("  template <typename R>")
        o.append("  __device__ __forceinline__ static void hrr(const R* __restrict__ acc, R* __restrict__ out,")
        o.append("      const R* AB, const R* CD) {")
        o.append("    (void)AB; (void)CD;")
        if lb == 0 and ld == 0:
            o.append(f"    #pragma unroll")
            o.append(f"    for (int x = 0; x < {NE * NF}; ++x) out[x] = acc[x];")
        else:
            o.append(f"    R hb[{ncart(la) * ncart(lb) * NF}];")
            o += ["    " + s for s in hlines]
        o.append("  }")
        o.append("};")
        o.append("")
    o.append("")
    o.append("// Cooperative schedules: node = (out | x0<<16, x1 | x2<<16, x3 | x4<<16,")
    o.append("// c0 | c1<<6 | c2<<12 | c3<<18 | c4<<24 | type<<30): out = c0*x0 + c1*x1 + c2*(x2 - c3*x3) + c4*x4,")
    o.append("// the c2 term present iff type bit 0, the c4 term iff type bit 1")
    o.append("// over slots (0..L = B[m]) and the coefficient vector; levels[k] = end of level k.")
    o.append("#define HF_COEF_NAMES \\")
    o.append("  " + " ".join(COEF_NAMES))
    o.append(f"#define HF_NCOEF {len(COEF_NAMES)}")
    o.append("template <class C> struct CoopTables;  // defined per class where its kernel is instantiated")
    for name, words, bounds, tgt in coop_tables:
        o.append(f"#ifdef HF_COOP_{name}")
        o.append(f"static __device__ const uint4 {name}_nodes[{len(words)}] = {{")
        for k in range(0, len(words), 4):
            o.append("  " + ", ".join("{%du,%du,%du,%du}" % w for w in words[k:k + 4]) + ",")
        o.append("};")
        o.append(f"static __device__ const int {name}_levels[{len(bounds)}] = {{{', '.join(map(str, bounds))}}};")
        o.append(f"static __device__ const unsigned short {name}_targets[{len(tgt)}] = {{{', '.join(map(str, tgt))}}};")
        o.append(f"template <> struct CoopTables<{name}> {{")
        o.append(f"  __device__ static const uint4* nodes() {{ return {name}_nodes; }}")
        o.append(f"  __device__ static const int* levels() {{ return {name}_levels; }}")
        o.append(f"  __device__ static const unsigned short* targets() {{ return {name}_targets; }}")
        o.append("};")
        o.append("#endif")
    o.append("}  // namespace hfgen")
    o.append("")
    o.append("// name, la, lb, lc, ld, VRR flops / primitive quartet, HRR flops / contracted quartet")
    o.append("#define HF_GEN_CLASS_TABLE(X) \\")
    for k, (name, la, lb, lc, ld, vf, hf) in enumerate(table):
        sep = " \\" if k + 1 < len(table) else ""
        o.append(f"  X({name}, {la}, {lb}, {lc}, {ld}, {vf}, {hf}){sep}")
    o.append("")
    return "\n".join(o)


def main():
    out = sys.argv[1]
    lmax = int(sys.argv[2]) if len(sys.argv) > 2 else 2
    txt = emit(lmax)
    try:
        old = open(out).read()
    except OSError:
        old = None
    if old != txt:
        with open(out, "w") as fh:
            fh.write(txt)


if __name__ == "__main__":
    main()
