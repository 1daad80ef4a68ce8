"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks
that the pins in ``oracle_pins.py`` catch every one of them.

The committed oracle source is never modified: each mutant is a text
substitution written to a temporary directory and compiled separately.
"""
import os

import pytest

import oracle
import oracle_pins as pins

ORACLE_DIR = os.path.dirname(oracle.__file__)
SOURCES = ["vct_oracle.c", "vct_voxelize.c", "vct_gbuffer.c"]

MUTANTS = {
    "texel centre dropped": ("double u = q[a] * nl - 0.5;", "double u = q[a] * nl;"),
    "x/z transposed in lookup": (
        "const double *v = lv + (((size_t)z * nl + y) * nl + x) * 4;",
        "const double *v = lv + (((size_t)x * nl + y) * nl + z) * 4;"),
    "printed colour line taken literally": (
        "for (int ch = 0; ch < 3; ++ch) c[ch] += cw * v[ch];",
        "for (int ch = 0; ch < 3; ++ch) c[ch] = alpha * c[ch] + cw * v[ch];"),
    "level from diameter / scene size": (
        "stencil(g->n, g->levels, q, log2(d / h0), &st);",
        "stencil(g->n, g->levels, q, log2(d / g->size), &st);"),
    "reflection sign": ("cs->dir[c][a] = view[a] - 2.0 * vn * nrm[a];",
                        "cs->dir[c][a] = view[a] + 2.0 * vn * nrm[a];"),
    "step ignores beta": ("alpha += wgt;\n    t += P->beta * d;", "alpha += wgt;\n    t += d;"),
    "mip divides by 4": ("dst[(((size_t)z * np + y) * np + x) * 4 + c] = s / 8.0;",
                         "dst[(((size_t)z * np + y) * np + x) * 4 + c] = s / 4.0;"),
    "level blend swapped": ("s->level_w[0] = 1.0 - f;\n  s->level_w[1] = f;",
                            "s->level_w[0] = f;\n  s->level_w[1] = 1.0 - f;"),
    "left-handed frame": ("cross3(nrm, T, B);", "cross3(T, nrm, B);"),
    "apex offset into the surface": (
        "cs->apex[a] = x[a] + P->normal_offset_voxels * h0 * nrm[a];",
        "cs->apex[a] = x[a] - P->normal_offset_voxels * h0 * nrm[a];"),
    "clamp-to-edge instead of border zero": (
        "continue; /* outside the grid: empty */",
        "{ x = x < 0 ? 0 : (x >= nl ? nl - 1 : x); y = y < 0 ? 0 : (y >= nl ? nl - 1 : y);"
        " z = z < 0 ? 0 : (z >= nl ? nl - 1 : z); }"),
    "adjoint drops Q": ("da += ga * s->trans * Q;", "da += ga * Q;"),
    "adjoint suffix not attenuated": (
        "R[ch] = (premul ? s->c[ch] : s->a * s->c[ch]) + (1.0 - s->a) * R[ch];",
        "R[ch] = (premul ? s->c[ch] : s->a * s->c[ch]) + R[ch];"),
    "premultiplied adjoint takes the straight colour weight": (
        "dc[ch] = gc[ch] * s->trans;", "dc[ch] = gc[ch] * s->trans * s->a;"),
    "premultiplied adjoint: opacity term sign": ("da -= gc[ch] * s->trans * R[ch];",
                                                 "da += gc[ch] * s->trans * R[ch];"),
    "occlusion fade left out of the adjoint": ("scatter_sample(g, gpyr, s, w, dc, da * s->sa);",
                                               "scatter_sample(g, gpyr, s, w, dc, da);"),
    "first-hit gradient to the first sample": (
        "if (r->hit) scatter_sample(g, gpyr, rec + r->steps - 1, w, gc, 0.0);",
        "if (r->hit) scatter_sample(g, gpyr, rec, w, gc, 0.0);"),
    "L_impl: dL/dD without Vis": ("dD[ch] = vis;", "dD[ch] = 1.0;"),
    "L_impl: dL/dVis without D": ("dV[ch] = D[ch] + direct[ch];", "dV[ch] = direct[ch];"),
    "L_vxct: direct light not occluded in the adjoint": ("dV[ch] = direct[ch];", "dV[ch] = 0.0;"),
    "L_vxct: specular ratio dropped in the adjoint": ("dS[ch] = alb[ch] * P->specular_str;",
                                                      "dS[ch] = alb[ch];"),
    "aniso: front and back of a pair swapped": (
        "const double *f = neg ? ch[1] : ch[0], *b = neg ? ch[0] : ch[1];",
        "const double *f = neg ? ch[0] : ch[1], *b = neg ? ch[1] : ch[0];"),
    "aniso: direction weights |w_a| instead of w_a^2": (
        "wa[a] = w[a] * w[a] / w2;", "wa[a] = fabs(w[a]) / sqrt(w2);"),
    "aniso: the opposite volume": ("dir[a] = 2 * a + (w[a] < 0.0 ? 1 : 0);",
                                   "dir[a] = 2 * a + (w[a] > 0.0 ? 1 : 0);"),
    "aniso: coarse levels from the isotropic level 0": (
        "pyr + orc_aniso_offset(n, l - 1, l == 1 ? 0 : d);", "pyr + orc_aniso_offset(n, l - 1, 0);"),
    "aniso: premultiplied colour stored": ("acc[c] += a > 0.0 ? pre / a : 0.0;", "acc[c] += pre;"),
    "aniso adjoint: opacity partial without (1 - a_b)": ("gf[3] = G[3] / 4.0 * (1.0 - ab);",
                                                          "gf[3] = G[3] / 4.0;"),
    "aniso adjoint: back colour partial without a_b": (
        "gb[c] = gC * (1.0 - af) * ab / alpha;", "gb[c] = gC * (1.0 - af) / alpha;"),
    "aniso adjoint: colour gradient through an empty pair": ("if (alpha > 0.0) {",
                                                             "if (alpha >= 0.0) {"),
    "aniso adjoint: front and back swapped": (
        "const size_t fi = neg ? ci[1] : ci[0], bi = neg ? ci[0] : ci[1];",
        "const size_t fi = neg ? ci[0] : ci[1], bi = neg ? ci[1] : ci[0];"),
    "aniso adjoint: scatter without the direction weight": (
        "scatter_level(&s->st, lk, gpyr + orc_aniso_offset(g->n, l, dir[a]), nl, wa[a], dc, da);",
        "scatter_level(&s->st, lk, gpyr + orc_aniso_offset(g->n, l, dir[a]), nl, 1.0, dc, da);"),
    "grace factor left out of the adjoint": (
        "double f = (P->flags & ORC_SPEC_GRACE) ? spec_grace(cs.dir[c], P) : 1.0;",
        "double f = 1.0;"),
    "mip adjoint weight": ("gp[(((size_t)(z / 2) * np + y / 2) * np + x / 2) * 4 + c] / 8.0;",
                           "gp[(((size_t)(z / 2) * np + y / 2) * np + x / 2) * 4 + c] / 4.0;"),
    "diffuse weight dropped": ("d[ch] += cs.weight[c] * r.c[ch];", "d[ch] += r.c[ch];"),
    "transmittance not stored": ("rec[k].trans = 1.0 - alpha;", "rec[k].trans = 1.0;"),
    "first-hit threshold": ("if (v[3] > 0.01) {", "if (v[3] > 0.001) {"),
    "smoothstep as a ramp": ("return t * t * (3.0 - 2.0 * t);", "return t;"),
    "angular grace without pi": ("double gn = acos(cosg) - 0.008 * pi * P->shininess;",
                                 "double gn = acos(cosg) - 0.008 * P->shininess;"),
    "light reflected the wrong way": ("R[a] = -l[a] + 2.0 * nl * n[a];",
                                      "R[a] = l[a] - 2.0 * nl * n[a];"),
    "direct light not occluded": (
        "out[ch] = alb[ch] * (P->diffuse_str * D[ch] + P->specular_str * S[ch]) + vis * direct[ch];",
        "out[ch] = alb[ch] * (P->diffuse_str * D[ch] + P->specular_str * S[ch]) + direct[ch];"),
    "top-left rule inverted": ("return ev < 0 || (ev == 0 && eu < 0);",
                               "return ev > 0 || (ev == 0 && eu > 0);"),
    "centre at the pixel corner": ("int64_t p[2] = {SUB * i + SUB / 2, SUB * j + SUB / 2};",
                                   "int64_t p[2] = {SUB * i, SUB * j};"),
    "depth rounded, not floored": ("int64_t k = floor_div(depth, SUB);",
                                   "int64_t k = floor_div(depth + SUB / 2, SUB);"),
    "dominant axis = smallest component": ("if (ax >= ay && ax >= az)",
                                           "if (ax <= ay && ax <= az)"),
    "first writer wins": ("stats[0] += 1;\n        owner_out[vox]",
                          "stats[0] += 1;\n        if (owner_out[vox]) continue;\n"
                          "        owner_out[vox]"),
    "back-facing light not clamped": ("if (lam < 0.0) lam = 0.0;", ""),
    "x-dominant swizzle transposed": ("au = 2;\n      av = 1;", "au = 1;\n      av = 2;"),
    "snap without the origin": ("float a = v - origin;", "float a = v;"),
    "premultiplied flag ignored": ("double cw = (P->flags & ORC_PREMUL) ? (1.0 - alpha) : wgt;",
                                   "double cw = wgt;"),
    "image rows not flipped": (
        "const float sy = (1.0f - (float)(2 * j + 1) / (float)H) * ty;",
        "const float sy = ((float)(2 * j + 1) / (float)H - 1.0f) * ty;"),
    "aspect ratio dropped": ("const float tx = (float)((double)tan_half * (double)W / (double)H);",
                             "const float tx = tan_half;"),
    "farthest hit wins": ("if (best < 0 || num * bden < bnum * den) {",
                          "if (best < 0 || num * bden > bnum * den) {"),
    "equal depth to the higher index": ("if (best < 0 || num * bden < bnum * den) {",
                                        "if (best < 0 || num * bden <= bnum * den) {"),
    "edges exclusive (det > 0)": ("hit = v[0] >= 0 && v[1] >= 0 && v[2] >= 0;",
                                  "hit = v[0] > 0 && v[1] > 0 && v[2] > 0;"),
    "edges exclusive (det < 0)": ("hit = v[0] <= 0 && v[1] <= 0 && v[2] <= 0;",
                                  "hit = v[0] < 0 && v[1] < 0 && v[2] < 0;"),
    "hits behind the camera": ("if (det > 0)\n        hit =", "if (v[0] + v[1] + v[2] > 0)\n        hit ="),
    "normal not turned to the camera": ("const double sgn = bsigned > 0 ? -1.0 : 1.0;",
                                        "const double sgn = 1.0;"),
    "camera frame snap without the origin": ("const float rel = v - origin;",
                                             "const float rel = v;"),
    "hit position without the frame origin": (
        "pos[3 * q + a] =\n          (double)frame_origin[a] + (", "pos[3 * q + a] =\n          ("),
}

CHECKS = [name for name in dir(pins) if name.startswith("check_")]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    srcs, hits = [], 0
    for fname in SOURCES:
        with open(os.path.join(ORACLE_DIR, fname)) as f:
            text = f.read()
        hits += text.count(old)
        src = tmp_path / fname
        src.write_text(text.replace(old, new))
        srcs.append(str(src))
    assert hits == 1, f"mutation anchor not unique/found: {old!r}"
    lib = oracle.load_library(oracle.compile_source(srcs, out_dir=str(tmp_path), tag="mutant"))
    caught = []
    with oracle.using(lib):
        for check in CHECKS:
            try:
                getattr(pins, check)()
            except AssertionError:
                caught.append(check)
    assert caught, f"no pin caught the planted mistake '{name}'"
