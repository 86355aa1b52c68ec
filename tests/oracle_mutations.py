#!/usr/bin/env python
"""Sensitivity of the oracle pins: plants one plausible mistake at a time in
a temporary copy of the oracle (the C reconstruction, the Python classifier
with its Adam optimiser, and the truth matching) and runs the oracle pins
(tests/test_oracle_*.py) against it.  Every mutant must fail at least one
pin, except the ones listed as equivalent (no observable effect).

    python tests/oracle_mutations.py        # a few minutes on the CPU

Not collected by pytest (too slow for the CPU suite).
"""
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in oracle/velo_oracle.c, replacement)
MUTANTS = [
    ("4-connectivity", "            int cc = c + dc, rr = r + dr;",
     "            if (dc != 0 && dr != 0) continue;\n            int cc = c + dc, rr = r + dr;"),
    ("centroid x without +1/2", "float lx = ((float)sc / (float)npix + 0.5f) * g->pitch;",
     "float lx = ((float)sc / (float)npix) * g->pitch;"),
    ("col/row axes swapped", "float x = g->sensor_ox[s] + cdx * lx + rdx * ly;",
     "float x = g->sensor_ox[s] + cdx * ly + rdx * lx;"),
    ("forward extrapolation sign", "float dzi = Z[i] - zl;", "float dzi = zl - Z[i];"),
    ("skip rule off by one", "if (w->skip[t] > p->max_skipped) w->active[t] = 0;",
     "if (w->skip[t] >= p->max_skipped) w->active[t] = 0;"),
    ("forwarded hits not marked used", "if (append[t] >= 0) used[append[t]] = 1;",
     "if (append[t] >= 0) used[append[t]] = 0;"),
    ("used middle hit allowed", "      if (used[b]) continue;\n      w->work[2]++;", "      w->work[2]++;"),
    ("used a allowed", "        if (used[a]) continue;", ""),
    ("used c allowed", "          if (used[c]) continue;", ""),
    ("seed extrapolation sign", "float dzc = Z[i] - Z[i + 1];", "float dzc = Z[i + 1] - Z[i];"),
    ("slope cut on x only", "if (fabsf(tx) > p->max_slope || fabsf(ty) > p->max_slope) continue;",
     "if (fabsf(tx) > p->max_slope) continue;"),
    ("slope cut on y only", "if (fabsf(tx) > p->max_slope || fabsf(ty) > p->max_slope) continue;",
     "if (fabsf(ty) > p->max_slope) continue;"),
    ("forwarding tie to the larger id", "(s == bs && (int32_t)h < best)", "(s == bs && (int32_t)h > best)"),
    ("seed tie to the larger c", "((int32_t)a == ba && (int32_t)c < bc)", "((int32_t)a == ba && (int32_t)c > bc)"),
    ("3-hit cut uses the seed cut", "keep = w->seed_s[t] < p->max_scatter_3hit",
     "keep = w->seed_s[t] < p->max_scatter_seed"),
    ("3-hit sharing checks two hits", "cnt[w->hits[t][1]] == 1 && cnt[w->hits[t][2]] == 1;",
     "cnt[w->hits[t][1]] == 1;"),
    ("long tracks from 5 hits", "if (w->n[t] >= 4) keep = 1;", "if (w->n[t] >= 5) keep = 1;"),
    ("scattering once per hit", "s.c11 = s.c11 + dm[k] * q_per_module;", "s.c11 = s.c11 + q_per_module;"),
    ("chi2 without measurement variance", "float R = sig2 + s.c00;", "float R = s.c00 + s.c00;"),
    ("beamline sign", "if (tt >= 1e-12f) zb = z - (fx.u * fx.tu + fy.u * fy.tu) / tt;",
     "if (tt >= 1e-12f) zb = z + (fx.u * fx.tu + fy.u * fy.tu) / tt;"),
    ("initial slope variance", "s.c11 = (2.0f * sig2) / (dz1 * dz1);", "s.c11 = sig2 / (dz1 * dz1);"),
    ("ndof", "*ndof = 2 * n - 4;", "*ndof = 2 * n - 3;"),
    ("scattering constant", "float kms = p->ms_coeff * 0.001f / p->pt_nominal;",
     "float kms = p->ms_coeff * 0.001f * p->pt_nominal;"),
    ("covariance update order", "    s.c10 = s.c10 - k1 * s.c00;\n    s.c00 = s.c00 - k0 * s.c00;",
     "    s.c00 = s.c00 - k0 * s.c00;\n    s.c10 = s.c10 - k1 * s.c00;"),
    ("per-track momentum ignored", "  if (p_track > 0.0f) sig_ms = (p->ms_coeff * 0.001f) / p_track;\n", ""),
    ("per-track kick grows with p", "sig_ms = (p->ms_coeff * 0.001f) / p_track;", "sig_ms = (p->ms_coeff * 0.001f) * p_track;"),
    ("prediction covariance", "s.c00 = s.c00 + dz * s.c10 + dz * c10n;\n    s.c10 = c10n;\n    s.c11 = s.c11 + dm[k]",
     "s.c00 = s.c00 + dz * c10n;\n    s.c10 = c10n;\n    s.c11 = s.c11 + dm[k]"),
]

# (name, text in oracle/mlp.py, replacement): the classifier's features and
# BF16 network
MUTANTS_MLP = [
    ("first-layer ReLU missing", "        h1[:, j] = bf16_round(np.maximum(acc, f32(0)))", "        h1[:, j] = bf16_round(acc)"),
    ("second-layer activation not rounded", "        h2j = bf16_round(np.maximum(acc, f32(0)))",
     "        h2j = np.maximum(acc, f32(0))"),
    ("inputs not rounded", "    x = bf16_round(normalise(f, mean, istd))", "    x = normalise(f, mean, istd)"),
    ("second-layer bias dropped", "        acc = np.full(n, b2[j], np.float32)", "        acc = np.zeros(n, np.float32)"),
    ("chi2 not per ndof", "    f[:, 0] = chi2 / np.asarray(ndof).astype(np.float32)", "    f[:, 0] = chi2"),
    ("eta argument", "        q = (f32(1.0) + s) / np.where(t > f32(1e-7), t, f32(1.0))",
     "        q = (f32(1.0) + t) / np.where(t > f32(1e-7), s, f32(1.0))"),
    ("phi arguments swapped", "    f[:, 8] = atan2_f32(ty, tx)", "    f[:, 8] = atan2_f32(tx, ty)"),
    ("missed modules off by one", "    f[:, 9] = ((mf - ml + 1) - n).astype(np.float32)",
     "    f[:, 9] = ((mf - ml) - n).astype(np.float32)"),
    ("log series coefficient 1/5 as 1/7", "    for c in (_INV[4], _INV[3], _INV[2], _INV[1], _INV[0]):\n        p = p * v + c\n    r =",
     "    for c in (_INV[4], _INV[3], _INV[3], _INV[1], _INV[0]):\n        p = p * v + c\n    r ="),
    ("second-layer sum order reversed", "        for k in range(N_H):\n            acc = acc + W2[j, k] * h1[:, k]",
     "        for k in reversed(range(N_H)):\n            acc = acc + W2[j, k] * h1[:, k]"),
    ("output bias dropped", "    out = np.full(n, b3[0], np.float32)\n", "    out = np.zeros(n, np.float32)\n"),
    ("atan reduction constant dropped", "    a = np.where(big, a + _PI6, a).astype(np.float32)",
     "    a = np.where(big, a, a).astype(np.float32)"),
    ("BF16 ties away from zero", "    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16", "    b = (b + 0x8000) >> 16"),
    ("standardisation divides", "    return ((np.asarray(f, np.float32) - mean.astype(np.float32)) * istd.astype(np.float32))",
     "    return ((np.asarray(f, np.float32) - mean.astype(np.float32)) / istd.astype(np.float32))"),
    ("first-layer sum order reversed", "        for i in range(N_IN):\n            acc = acc + W1[j, i] * x[:, i]",
     "        for i in reversed(range(N_IN)):\n            acc = acc + W1[j, i] * x[:, i]"),
    # the optimiser of the training step
    ("Adam betas swapped", "self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps",
     "self.lr, self.b1, self.b2, self.eps = lr, b2, b1, eps"),
    ("Adam first moment not bias-corrected", "        mh = self.m / (1 - self.b1 ** self.t)", "        mh = self.m"),
    ("Adam second moment not bias-corrected", "        vh = self.v / (1 - self.b2 ** self.t)", "        vh = self.v"),
    ("Adam eps inside the square root", "self.w -= self.lr * mh / (np.sqrt(vh) + self.eps)",
     "self.w -= self.lr * mh / np.sqrt(vh + self.eps)"),
    ("Adam second moment of |g|", "(1 - self.b2) * g * g", "(1 - self.b2) * np.abs(g)"),
]

# (name, text in oracle/metrics.py, replacement): truth matching
MUTANTS_METRICS = [
    ("match fraction 0.6", "MATCH_FRACTION = 0.7", "MATCH_FRACTION = 0.6"),
    ("reconstructible from 2 modules", "    return cnt >= 3", "    return cnt >= 2"),
    ("clone rate over all tracks", "clone_rate=float(len(matched) - n_unique) / len(matched)",
     "clone_rate=float(len(matched) - n_unique) / n_tracks"),
    ("efficiency counts every found particle", "n_found = int((found & rec).sum())", "n_found = int(found.sum())"),
    ("cluster label ties to the larger index", "order = np.lexsort((uniq[:, 1], -cnt, uniq[:, 0]))",
     "order = np.lexsort((-uniq[:, 1], -cnt, uniq[:, 0]))"),
    ("repeated pixel takes the larger index", "order = np.lexsort((labk, u))", "order = np.lexsort((-labk, u))"),
    ("ghosts counted from matched tracks", "ghost_rate=float((match < 0).sum()) / n_tracks",
     "ghost_rate=float((match >= 0).sum()) / n_tracks"),
]

# (name, text in oracle/pv_oracle.c, replacement): primary-vertex finding
MUTANTS_PV = [
    ("Tukey weight not squared", "  float u = 1.0f - chi2 / cut;\n  return u * u;", "  float u = 1.0f - chi2 / cut;\n  return u;"),
    ("weight without the share", "float w = (t * t) / tsum[i];", "float w = t;"),
    ("position variance without the correlation",
     "return (cpp + dz * (cpt + cpt)) + (dz * dz) * ctt;", "return cpp + (dz * dz) * ctt;"),
    ("z step sign", "float dz = ((px * V->bx + py * V->by) - V->bt) / D;",
     "float dz = (V->bt - (px * V->bx + py * V->by)) / D;"),
    ("x variance without the z term", "o[3] = 1.0f / V->sxx + (px * px) / D;", "o[3] = 1.0f / V->sxx;"),
    ("merge rule off", "if (fabsf(vtx[u].z - vtx[v].z) < p->merge_dz &&", "if (fabsf(vtx[u].z - vtx[v].z) < 0.0f &&"),
    ("equal peaks: the larger bin dominates", "(win[c] == win[b] && c < b)", "(win[c] == win[b] && c > b)"),
    ("beam-axis cut on x only", "if (!(s[0] * s[0] + s[1] * s[1] < p->max_r2)) continue;",
     "if (!(s[0] * s[0] < p->max_r2)) continue;"),
    ("histogram bin rounded", "hist[(uint32_t)u] += 1;", "hist[(uint32_t)(u + 0.5f)] += 1;"),
    ("no suppression of nearby seeds", "if (dominated) continue;", "if (0) continue;"),
    ("peak at the first bin of its run", "  return b == p0 + (p1 - p0) / 2;", "  return b == p0;"),
    ("shoulders are peaks", "  if (p0 > 0 && win[p0 - 1] > win[b]) return 0;\n", ""),
    ("kept with any weight", "int ok = V->sxx > 0.0f && V->syy > 0.0f && V->sw >= p->min_weight;",
     "int ok = V->sxx > 0.0f && V->syy > 0.0f;"),
]

# Mutants that cannot change any output:
#   - duplicates kept in the sorted key list: the flood fill still visits
#     (and counts) every pixel position once;
#   - a seed's a hit not marked used: its module never takes part in a later
#     seed, and forwarding does not look at used flags.
EQUIVALENT = [
    # the last term of the log series is below float32 resolution
    # (2 u^11 / 11 < 8e-10 relative for |u| <= 0.172)
    ("log series u^11 term dropped", "    for c in (_INV[4], _INV[3], _INV[2], _INV[1], _INV[0]):\n        p = p * v + c\n    r =",
     "    for c in (_INV[3], _INV[2], _INV[1], _INV[0]):\n        p = p * v + c\n    r =", "mlp.py"),
    ("duplicates kept", "if (i == 0 || keys[i] != keys[i - 1]) keys[nu++] = keys[i];", "keys[nu++] = keys[i];"),
    ("seed a not marked used", "used[seeds[k][0]] = 1; used[seeds[k][1]] = 1;", "used[seeds[k][1]] = 1;"),
]

PINS = ["tests/test_oracle_tracking.py", "tests/test_oracle_cluster.py", "tests/test_oracle_fit.py",
        "tests/test_oracle_mlp.py", "tests/test_oracle_metrics.py", "tests/test_oracle_pv.py"]


def run(name, old, new, target="velo_oracle.c"):
    with tempfile.TemporaryDirectory() as d:
        for sub in ("oracle", "velo_synth", "tests"):
            shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                            ignore=shutil.ignore_patterns("*.so", "__pycache__"))
        shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
        p = os.path.join(d, "oracle", target)
        s = open(p).read()
        assert s.count(old) == 1, name
        open(p, "w").write(s.replace(old, new))
        r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-q", "-x", "-p", "no:cacheprovider"], cwd=d,
                           capture_output=True, text=True, timeout=900)
        failed = [ln.split("::")[-1] for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
        return r.returncode != 0, failed


def main() -> int:
    missed = []
    for name, old, new in MUTANTS:
        caught, failed = run(name, old, new)
        print(f"{'caught' if caught else 'MISSED'}: {name:34s} {failed[:1]}", flush=True)
        if not caught:
            missed.append(name)
    for name, old, new in MUTANTS_MLP:
        caught, failed = run(name, old, new, "mlp.py")
        print(f"{'caught' if caught else 'MISSED'}: {name:34s} {failed[:1]}", flush=True)
        if not caught:
            missed.append(name)
    for name, old, new in MUTANTS_METRICS:
        caught, failed = run(name, old, new, "metrics.py")
        print(f"{'caught' if caught else 'MISSED'}: {name:34s} {failed[:1]}", flush=True)
        if not caught:
            missed.append(name)
    for name, old, new in MUTANTS_PV:
        caught, failed = run(name, old, new, "pv_oracle.c")
        print(f"{'caught' if caught else 'MISSED'}: {name:34s} {failed[:1]}", flush=True)
        if not caught:
            missed.append(name)
    for name, old, new, *target in EQUIVALENT:
        caught, _ = run(name, old, new, *target)
        print(f"{'caught' if caught else 'no effect'}: {name} (equivalent)", flush=True)
    total = len(MUTANTS) + len(MUTANTS_MLP) + len(MUTANTS_METRICS) + len(MUTANTS_PV)
    print(f"{total - len(missed)} of {total} mutants caught")
    return 1 if missed else 0


if __name__ == "__main__":
    sys.exit(main())
