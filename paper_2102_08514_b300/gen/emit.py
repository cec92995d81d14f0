"""Emit the generator's tables as a C++ header consumed by the CUDA kernels, plus JSON metadata.

    python -m paper_2102_08514_b300.gen.emit            # (re)writes csrc/generated/

The header holds, per built-in spline, a struct of `static constexpr` tables: the coset shifts, the
chamber planes and the sigma table (Sec. 4.2), and per piece its anchor, its gather stencil and the
nonzero entries of its coefficient matrix A (monomial x site) in the nested-Horner monomial layout.
Values are the exact rationals rounded once to FP32 and written as hexadecimal literals.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
from fractions import Fraction as Fr

import numpy as np

from .catalog import CATALOG, VORONOI
from .pieces import analyse, analyse_voronoi, horner_order, n_monomials, sec42_compression

GEN_VERSION = 1
HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(os.path.dirname(HERE), "csrc", "generated")
# splines whose FP16 / BF16 coefficient-storage kernels are compiled (the 4-D spline's kernels are
# large, so only its FP32 variant is built)
HALF_STORAGE = {"bcc_linear", "bcc_quintic", "fcc_6dir", "cc_7dir", "bcc_quartic", "cc_linear_rd", "cc_voronoi1",
                "cc_voronoi2", "cc_voronoi3", "bcc_voronoi1", "fcc_voronoi1"}
# the 3-D splines compiled into the persistent batched kernel: few pieces and registers, so that
# one of them does not lower the kernel's occupancy for the others
BATCH_3D = {"bcc_linear", "bcc_quintic", "fcc_6dir", "cc_7dir", "bcc_quartic", "cc_linear_rd", "cc_voronoi1",
            "cc_voronoi2"}
# sigma has 2^Q entries: up to 64 of them are packed as 4-bit piece indices into 64-bit constants
# (K <= 15), larger tables are byte arrays in device memory (Q <= 12)
MAX_PIECES, MAX_PACKED, MAX_Q = 15, 64, 12


def dense_pieces(T, nz_lists) -> bool:
    """Splines for which dense device tables of A_j are emitted (one shared loop over the sites
    instead of one unrolled code block per piece): many pieces with many nonzeros, whose unrolled
    code does not fit the instruction caches.  The binned rays kernel uses them; the binned
    evaluation of random queries keeps the unrolled code (measured faster)."""
    return len(T.pieces) >= 8 and max(len(z) for z in nz_lists) >= 400


def analyse_entry(name):
    """The generator's tables for a built-in name (box spline or Voronoi spline)."""
    if name in VORONOI:
        L, gens, order = VORONOI[name]
        return analyse_voronoi(name, L, gens, order)
    L, xi = CATALOG[name]
    return analyse(name, L, xi)


def f32_hex(v) -> str:
    x = float(np.float32(float(Fr(v))))
    if x == 0.0:
        return "0.0f"
    return f"{x.hex()}f"


def horner_fma_count(s, d):
    """FMAs of the nested Horner evaluation of a dense polynomial of degree d in s variables."""
    if s == 0:
        return 0
    return sum(horner_fma_count(s - 1, d - k) for k in range(d + 1)) + d


def horner_grad_fma_count(s, d):
    """FMAs of the nested Horner evaluation carrying the value and all s partial derivatives."""
    if s == 0:
        return 0
    inner = sum(horner_grad_fma_count(s - 1, d - k) for k in range(d + 1))
    # per step of the outer Horner: value (1), d/dt_1 (1), and s-1 inner partials (s-1)
    return inner + d * (s + 1)


def _block_off(nv, d, k):
    return sum(n_monomials(nv - 1, d - kk) for kk in range(k))


def horner_ops(nz, s, d, off=0):
    """(nonzero?, FP32 operations) of the kernels' nested Horner evaluation of a polynomial in s
    variables of degree d whose coefficients b[off ..] (nested-Horner layout) are structurally
    zero outside the index set nz.  A step acc * t + p costs one FMA when both are nonzero, one
    multiply when only acc is, nothing when acc is zero (acc = p); zero coefficients are never
    loaded or added."""
    if s == 0:
        return off in nz, 0
    acc, ops = horner_ops(nz, s - 1, 0, off + _block_off(s, d, d))
    for k in range(d - 1, -1, -1):
        p, o = horner_ops(nz, s - 1, d - k, off + _block_off(s, d, k))
        ops += o
        if acc:
            ops += 1
        elif p:
            acc = True
    return acc, ops


def horner_grad_ops(nz, s, d, off=0):
    """(value nonzero?, [partials nonzero?], FP32 operations) of the nested Horner evaluation
    that carries the s partial derivatives, with the same structural-zero rule as horner_ops."""
    if s == 0:
        return off in nz, [], 0
    v, g, ops = horner_grad_ops(nz, s - 1, 0, off + _block_off(s, d, d))
    g0, gr = False, list(g)

    def step(a, b):
        # a * t + b: one operation unless a is zero; the result is nonzero if either is
        return (a or b), (1 if a else 0)

    for k in range(d - 1, -1, -1):
        pv, pg, o = horner_grad_ops(nz, s - 1, d - k, off + _block_off(s, d, k))
        ops += o
        if k == d - 1:
            g0 = v                                   # d/dt_1 of the leading block: a copy
        else:
            g0, o = step(g0, v)
            ops += o
        v, o = step(v, pv)
        ops += o
        for j in range(s - 1):
            gr[j], o = step(gr[j], pg[j])
            ops += o
    return v, [g0] + gr, ops


def op_counts(s, degree, M, pieces):
    """FP32 operations per query of one value and of one value + gradient evaluation: per coset
    and piece (weighted by the piece's share of the fold chamber) the nonzeros of A_j (b = A_j c)
    plus the Horner steps on structurally nonzero data, and the sums over the M cosets.
    pieces: (volume fraction, [(site, monomial index, value)]) per piece."""
    val = grad = 0.0
    for w, z in pieces:
        nz = {a for _, a, _ in z}
        val += w * (len(z) + horner_ops(nz, s, degree)[1])
        grad += w * (len(z) + horner_grad_ops(nz, s, degree)[2])
    return M * val + (M - 1), M * grad + (M - 1) * (1 + s)


def piece_volumes(T):
    from scipy.spatial import ConvexHull
    vols = []
    for pc in T.pieces:
        V = np.array([[float(a) for a in v] for v in pc.verts])
        vols.append(ConvexHull(V).volume)
    tot = sum(vols)
    return [v / tot for v in vols]


def _arr(vals, fmt=str):
    return "{" + ", ".join(fmt(v) for v in vals) + "}"


def emit_struct(T, half_storage: bool = True) -> tuple[str, dict]:
    s = T.s
    order = horner_order(s, T.degree)
    index = {e: i for i, e in enumerate(order)}
    nmon = n_monomials(s, T.degree)
    K = len(T.pieces)
    nsmax = max(len(pc.sites) for pc in T.pieces)
    nz_lists = []
    for pc in T.pieces:
        nz = []
        for m, P in enumerate(pc.polys):
            for e, v in sorted(P.c.items(), key=lambda kv: index[kv[0]]):
                nz.append((m, index[e], v))
        nz_lists.append(nz)
    nnzmax = max(len(z) for z in nz_lists)
    Q = len(T.planes)
    vols = piece_volumes(T)
    hv = horner_fma_count(s, T.degree)
    hg = horner_grad_fma_count(s, T.degree)
    M = len(T.cosets)
    fma_value, fma_grad = op_counts(s, T.degree, M, list(zip(vols, nz_lists)))
    lookups = M * sum(w * len(pc.sites) for w, pc in zip(vols, T.pieces))

    L = [f"// ---- spline {T.name}"]
    if T.r > MAX_PACKED:
        # sigma as a byte table in device memory (read through the read-only cache)
        L.append(f"static __device__ const unsigned char {T.name}_sigma_tab[{T.r}] = {_arr(T.sigma)};")
    dense = dense_pieces(T, nz_lists)
    if dense:
        # A_j dense, site-major, monomials padded to a multiple of 4 (float4 loads), zero columns
        # past the piece's own sites; the sites, their count and the anchors per piece
        nm4 = (nmon + 3) // 4
        vals = []
        for j, z in enumerate(nz_lists):
            A = [[Fr(0)] * (nm4 * 4) for _ in range(nsmax)]
            for m, a, v in z:
                A[m][a] = v
            for row in A:
                vals.extend(row)
        L.append(f"static __device__ const float __align__(16) {T.name}_dense_a[{len(vals)}] = "
                 f"{_arr(vals, f32_hex)};")
        sites = []
        for pc in T.pieces:
            for m in range(nsmax):
                sites.extend(pc.sites[m] if m < len(pc.sites) else [0] * s)
        L.append(f"static __device__ const signed char {T.name}_dense_site[{len(sites)}] = {_arr(sites)};")
        L.append(f"static __device__ const int {T.name}_dense_ns[{K}] = {_arr([len(pc.sites) for pc in T.pieces])};")
        L.append(f"static __device__ const float {T.name}_dense_anchor[{K * s}] = "
                 f"{_arr([a for pc in T.pieces for a in pc.anchor], f32_hex)};")
    L.append(f"struct {T.name} {{")
    L.append(f'    static constexpr const char* NAME = "{T.name}";')
    L.append(f"    static constexpr int S = {s}, NXI = {len(T.xi[0])}, M = {M}, D = {T.D}, DETL = {T.det_l};")
    L.append(f"    static constexpr int K = {K}, Q = {Q}, R = {T.r}, DEG = {T.degree}, NMON = {nmon}, HALO = {T.halo};")
    L.append(f"    static constexpr int NSMAX = {nsmax}, NNZMAX = {nnzmax}, FOLD = {T.fold};")
    L.append(f"    static constexpr int KIND = {T.kind};  // 0: box spline M_XI; n: Voronoi spline V_n, XI = 2 G")
    L.append(f"    static constexpr int SMOOTH = {T.smooth};  // phi is in C^SMOOTH")
    L.append(f"    static constexpr bool HALF_STORAGE = {'true' if half_storage else 'false'};  // FP16/BF16 kernels built")
    L.append(f"    static constexpr int XI[S][NXI] = {_arr([_arr(r) for r in T.xi])};")
    L.append(f"    static constexpr int LMAT[S][S] = {_arr([_arr(r) for r in T.L])};")
    L.append(f"    static constexpr int COSET[M][S] = {_arr([_arr(c) for c in T.cosets])};")
    if Q:
        L.append(f"    static constexpr int PLANE_P[Q][S] = {_arr([_arr(p) for p, _ in T.planes])};")
        L.append(f"    static constexpr float PLANE_E[Q] = {_arr([e for _, e in T.planes], f32_hex)};")
    else:
        L.append("    static constexpr int PLANE_P[1][S] = {};")
        L.append("    static constexpr float PLANE_E[1] = {0.0f};")
    L.append(f"    static constexpr int SIGMA[R] = {_arr(T.sigma)};")
    if T.r > MAX_PACKED:
        L.append(f"    __device__ static unsigned sigma_at(unsigned q) {{ return __ldg(&{T.name}_sigma_tab[q]); }}")
    L.append(f"    static constexpr bool DENSE = {'true' if dense else 'false'};  // dense A_j tables emitted")
    if dense:
        L.append(f"    __device__ static const float4 *dense_a(int j) {{ return reinterpret_cast<const float4 *>("
                 f"{T.name}_dense_a) + j * {nsmax * ((nmon + 3) // 4)}; }}")
        L.append(f"    __device__ static const signed char *dense_site(int j) {{ return {T.name}_dense_site + j * {nsmax * s}; }}")
        L.append(f"    __device__ static int dense_ns(int j) {{ return __ldg(&{T.name}_dense_ns[j]); }}")
        L.append(f"    __device__ static const float *dense_anchor(int j) {{ return {T.name}_dense_anchor + j * {s}; }}")
    L.append(f"    static constexpr int NS[K] = {_arr([len(pc.sites) for pc in T.pieces])};")
    L.append(f"    static constexpr int NNZ[K] = {_arr([len(z) for z in nz_lists])};")
    L.append(f"    static constexpr float ANCHOR[K][S] = {_arr([_arr(pc.anchor, f32_hex) for pc in T.pieces])};")
    sites = []
    for pc in T.pieces:
        rows = [_arr(g) for g in pc.sites] + [_arr([0] * s)] * (nsmax - len(pc.sites))
        sites.append(_arr(rows))
    L.append(f"    static constexpr signed char SITE[K][NSMAX][S] = {_arr(sites)};")
    # nonzeros of A_j as a type list nz<site, monomial, value, first write of b[monomial],
    # first entry of its site, last entry of its site>, grouped by site
    for j, z in enumerate(nz_lists):
        seen = set()
        ents = []
        for idx, (m, a, v) in enumerate(z):
            sf = int(idx == 0 or z[idx - 1][0] != m)
            sl = int(idx == len(z) - 1 or z[idx + 1][0] != m)
            ents.append(f"nz<{m}, {a}, {f32_hex(v)}, {int(a not in seen)}, {sf}, {sl}>")
            seen.add(a)
        body = ",\n        ".join(", ".join(ents[i:i + 3]) for i in range(0, len(ents), 3))
        L.append(f"    using NZ{j} = nzlist<\n        {body}>;")
    L.append(f"    template <int J> using NZL = typename pick<J, {', '.join(f'NZ{j}' for j in range(K))}>::type;")
    # the same nonzeros split by outer Horner block k (monomials t_1^k * (t_2..t_s)^beta), with
    # monomial indices local to the block: NZB<J, k> drives the block-by-block evaluation
    deg = T.degree
    offs = [sum(n_monomials(s - 1, deg - kk) for kk in range(k)) for k in range(deg + 2)]
    for j, z in enumerate(nz_lists):
        blists = []
        for k in range(deg + 1):
            seen = set()
            ents = []
            for m, a, v in sorted(((m, a, v) for m, a, v in z if offs[k] <= a < offs[k + 1]), key=lambda e: (e[0], e[1])):
                ents.append(f"nz<{m}, {a - offs[k]}, {f32_hex(v)}, {int(a not in seen)}, 0, 0>")
                seen.add(a)
            body = ",\n        ".join(", ".join(ents[i:i + 3]) for i in range(0, len(ents), 3))
            L.append(f"    using NZB{j}_{k} = nzlist<{chr(10) + '        ' + body if ents else ''}>;")
            blists.append(f"NZB{j}_{k}")
        L.append(f"    using NZBL{j} = blocks<{', '.join(blists)}>;")
    L.append(f"    template <int J, int B> using NZB = typename pick_block<B, typename pick<J, {', '.join(f'NZBL{j}' for j in range(K))}>::type>::type;")
    L.append(f"    static constexpr double FMA_VALUE = {fma_value!r}, FMA_GRAD = {fma_grad!r}, LOOKUPS = {lookups!r};")
    L.append("};")

    meta = dict(name=T.name, kind=T.kind, smooth=T.smooth, s=s, L=T.L, xi=T.xi, det_l=T.det_l, D=T.D, cosets=T.cosets, fold=T.fold,
                degree=T.degree, n_monomials=nmon, halo=T.halo, r=T.r, sigma=T.sigma,
                planes=[[list(p), str(e)] for p, e in T.planes],
                r_sec42=sec42_compression([pc.code for pc in T.pieces], len(T.planes)),
                pieces=[dict(anchor=[str(a) for a in pc.anchor], sites=pc.sites, code=pc.code,
                             nnz=len(z), volume_fraction=w,
                             vertices=[[str(a) for a in v] for v in pc.verts],
                             ineqs=[[list(map(str, a)), str(b)] for a, b in pc.ineqs],
                             polys=[{",".join(map(str, e)): str(v) for e, v in P.c.items()} for P in pc.polys])
                        for pc, z, w in zip(T.pieces, nz_lists, vols)],
                fma_value=fma_value, fma_grad=fma_grad, lookups=lookups,
                horner_fma=hv, horner_grad_fma=hg)
    return "\n".join(L), meta


def recount(struct_text: str, meta: dict) -> tuple[str, dict]:
    """A spline's emitted struct and metadata with the operation counts recomputed from the
    metadata's exact polynomials (the counts are the only change)."""
    s, deg = meta["s"], meta["degree"]
    index = {e: i for i, e in enumerate(horner_order(s, deg))}
    pieces = []
    for pc in meta["pieces"]:
        z = [(m, index[tuple(int(v) for v in e.split(","))], Fr(v))
             for m, P in enumerate(pc["polys"]) for e, v in P.items()]
        pieces.append((pc["volume_fraction"], z))
    fv, fg = op_counts(s, deg, len(meta["cosets"]), pieces)
    meta = dict(meta, fma_value=fv, fma_grad=fg)
    lines = struct_text.split("\n")
    for i, ln in enumerate(lines):
        if "static constexpr double FMA_VALUE" in ln:
            lookups = ln.split("LOOKUPS = ")[1].rstrip(";")
            lines[i] = f"    static constexpr double FMA_VALUE = {fv!r}, FMA_GRAD = {fg!r}, LOOKUPS = {lookups};"
    return "\n".join(lines), meta


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=OUT_DIR)
    ap.add_argument("names", nargs="*", default=list(CATALOG) + list(VORONOI))
    ap.add_argument("--update", nargs="+", default=None, metavar="NAME",
                    help="re-analyse only these splines; take the others from the current output")
    ap.add_argument("--recount", action="store_true",
                    help="recompute only the operation counts of the current output (no re-analysis)")
    args = ap.parse_args(argv)
    if args.recount:
        args.update = ["__none__"]
    os.makedirs(args.out, exist_ok=True)
    old_structs, old_metas = {}, {}
    if args.update:
        with open(os.path.join(args.out, "splines.h")) as f:
            hdr_text = f.read()
        for block in hdr_text.split("\n// ---- spline ")[1:]:
            name = block.split("\n", 1)[0].strip()
            old_structs[name] = "// ---- spline " + block[:block.index("\n};") + 3]
        with open(os.path.join(args.out, "splines.json")) as f:
            old_metas = json.load(f)["splines"]
    structs, metas = [], {}
    for name in args.names:
        if args.update and name not in args.update and name in old_structs and name in old_metas:
            st, meta = old_structs[name], old_metas[name]
            if args.recount:
                st, meta = recount(st, meta)
            structs.append(st)
            metas[name] = meta
            continue
        T = analyse_entry(name)
        if len(T.pieces) > MAX_PIECES or len(T.planes) > MAX_Q:
            raise ValueError(f"{name}: {len(T.pieces)} pieces / {len(T.planes)} planes exceed the kernels' sigma table")
        # the kernels' FP32 plane test is within 2^-19 of exact for |p_a| <= 1, |e| <= 4 (they
        # recompute exactly below 2^-17)
        if any(abs(a) > 1 for p_, _ in T.planes for a in p_) or any(abs(e) > 4 for _, e in T.planes):
            raise ValueError(f"{name}: plane coefficients outside the kernels' exact-test bound")
        text, meta = emit_struct(T, half_storage=name in HALF_STORAGE)
        structs.append(text)
        metas[name] = meta
    body = "\n\n".join(structs)
    digest = hashlib.sha256(body.encode()).hexdigest()[:16]
    hdr = [
        "// Generated by paper_2102_08514_b300/gen/emit.py from the exact rational analysis of each",
        "// spline (pieces, stencils, polynomial coefficients rounded once to FP32). Do not edit.",
        f"// generator version {GEN_VERSION}, table digest {digest}",
        "#pragma once",
        "",
        "namespace interp_gen {",
        "",
        "// one nonzero A[mon][site] = val of a piece's coefficient matrix; FIRST: first write of b[mon];",
        "// SFIRST / SLAST: first / last nonzero of its site (the list is grouped by site)",
        "template <int SITE, int MON, float VAL, int FIRST, int SFIRST, int SLAST> struct nz {};",
        "template <class... Z> struct nzlist { static constexpr int size = sizeof...(Z); };",
        "template <int J, class T0, class... Ts> struct pick { using type = typename pick<J - 1, Ts...>::type; };",
        "template <class T0, class... Ts> struct pick<0, T0, Ts...> { using type = T0; };",
        "template <class... Bs> struct blocks {};",
        "template <int K, class BL> struct pick_block;",
        "template <int K, class... Bs> struct pick_block<K, blocks<Bs...>> { using type = typename pick<K, Bs...>::type; };",
        "",
        body,
        "",
        "}  // namespace interp_gen",
        "",
        "// X-macro over every built-in spline: X(struct name)",
        "#define INTERP_GEN_SPLINES(X) " + " ".join(f"X({n})" for n in args.names),
        "// the 3-D splines of the persistent batched kernel (comma-separated); other handles of a",
        "// batch run their own evaluation launch",
        "#define INTERP_GEN_BATCH_3D " + ", ".join(f"interp_gen::{n}" for n in args.names if n in BATCH_3D),
        "#define INTERP_GEN_BATCH_NAMES_3D " + ", ".join(f'"{n}"' for n in args.names if n in BATCH_3D),
        f'#define INTERP_GEN_DIGEST "{digest}"',
        "",
    ]
    with open(os.path.join(args.out, "splines.h"), "w") as f:
        f.write("\n".join(hdr))
    with open(os.path.join(args.out, "splines.json"), "w") as f:
        json.dump(dict(version=GEN_VERSION, digest=digest, splines=metas), f, indent=1)
    print(f"wrote {len(args.names)} splines, digest {digest}")


if __name__ == "__main__":
    main()
