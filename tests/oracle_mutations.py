#!/usr/bin/env python
"""Sensitivity of the oracle pins: plants one plausible mistake at a time in
a temporary copy of the oracle (C source) and runs the oracle pins
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
    ("used middle hit allowed", "      if (used[b]) continue;\n      int32_t ba = -1", "      int32_t ba = -1"),
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
    ("prediction covariance", "s.c00 = s.c00 + dz * s.c10 + dz * c10n;\n    s.c10 = c10n;\n    s.c11 = s.c11 + dm[k]",
     "s.c00 = s.c00 + dz * c10n;\n    s.c10 = c10n;\n    s.c11 = s.c11 + dm[k]"),
]

# Mutants that cannot change any output:
#   - duplicates kept in the sorted key list: the flood fill still visits
#     (and counts) every pixel position once;
#   - a seed's a hit not marked used: its module never takes part in a later
#     seed, and forwarding does not look at used flags.
EQUIVALENT = [
    ("duplicates kept", "if (i == 0 || keys[i] != keys[i - 1]) keys[nu++] = keys[i];", "keys[nu++] = keys[i];"),
    ("seed a not marked used", "used[seeds[k][0]] = 1; used[seeds[k][1]] = 1;", "used[seeds[k][1]] = 1;"),
]

PINS = ["tests/test_oracle_tracking.py", "tests/test_oracle_cluster.py", "tests/test_oracle_fit.py",
        "tests/test_oracle_mlp.py"]


def run(name, old, new):
    with tempfile.TemporaryDirectory() as d:
        for sub in ("oracle", "velo_synth", "tests"):
            shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                            ignore=shutil.ignore_patterns("*.so", "__pycache__"))
        shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
        p = os.path.join(d, "oracle", "velo_oracle.c")
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
    for name, old, new in EQUIVALENT:
        caught, _ = run(name, old, new)
        print(f"{'caught' if caught else 'no effect'}: {name} (equivalent)", flush=True)
    print(f"{len(MUTANTS) - len(missed)} of {len(MUTANTS)} mutants caught")
    return 1 if missed else 0


if __name__ == "__main__":
    sys.exit(main())
