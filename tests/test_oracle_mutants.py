"""Planted mistakes: each test copies the oracle's C sources, plants one
plausible mistake (a wrong coefficient or sign, a dropped term, an index off
by one, a swapped operand, a wrong constant), builds that copy and runs the
oracle's pin tests against it (ORACLE_LIBRARY).  The pins must fail for every
mistake, so they pin the oracle to the paper and the mathematics rather than
to itself.  The unmutated copy passes the same pins.  All on the CPU."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
STENCIL, GRADIENT, CODEC = "tests/test_oracle_stencil.py", "tests/test_oracle_gradient.py", "tests/test_oracle_codec.py"
BATCH = "tests/test_oracle_batch.py"

# (id, source file, text, replacement, pin file expected to catch it)
MUTANTS = [
    ("laplacian-coefficient-sign", "fwi_oracle.c", "-1.0 / 5.0, 8.0 / 315.0", "1.0 / 5.0, 8.0 / 315.0", STENCIL),
    ("laplacian-dropped-z-term", "fwi_oracle.c",
     "          acc += OC[r] * (oc_at(u, g, x, y, z + r) + oc_at(u, g, x, y, z - r));\n", "", STENCIL),
    ("laplacian-neighbour-index", "fwi_oracle.c", "(oc_at(u, g, x + r, y, z) + oc_at(u, g, x - r, y, z))",
     "(oc_at(u, g, x + r, y, z) + oc_at(u, g, x + r, y, z))", STENCIL),
    ("damping-sign", "fwi_oracle.c", "double am = m[i] * idt2 - sig[i] / (2.0 * g->dt);",
     "double am = m[i] * idt2 + sig[i] / (2.0 * g->dt);", STENCIL),
    ("sponge-profile-power", "fwi_oracle.c", "* (d / W) * (d / W)", "* (d / W)", STENCIL),
    ("source-one-step-late", "fwi_oracle.c", "double q = wavelet[n];", "double q = wavelet[n > 0 ? n - 1 : 0];",
     STENCIL),
    ("adjoint-residual-index", "fwi_oracle.c",
     "oc_step(g, m, sig, lcur, lnext, lnext, Lb, rc, resid + (long)(k - 1) * nrec, nrec);",
     "oc_step(g, m, sig, lcur, lnext, lnext, Lb, rc, resid + (long)(k > 1 ? k - 2 : 0) * nrec, nrec);", GRADIENT),
    ("gradient-residual-index", "fwi_oracle.c",
     "oc_step(g, m, sig, lcur, lnext, lnew, Lb, rc, resid + (long)(k - 1) * nrec, nrec);",
     "oc_step(g, m, sig, lcur, lnext, lnew, Lb, rc, resid + (long)(k > 1 ? k - 2 : 0) * nrec, nrec);", GRADIENT),
    ("imaging-sign", "fwi_oracle.c", "grad[i] -= weight * uk[i]", "grad[i] += weight * uk[i]", GRADIENT),
    ("subsampling-weight-dropped", "fwi_oracle.c", "grad[i] -= weight * uk[i]", "grad[i] -= uk[i]", GRADIENT),
    ("imaging-second-difference", "fwi_oracle.c", "(lnew[i] - 2.0 * lcur[i] + lnext[i])", "(lnew[i] - lnext[i])",
     GRADIENT),
    ("records-wrong-time-level", "fwi_oracle.c", "dsim[(long)s * nrec + r] = cur[rc[r]];",
     "dsim[(long)s * nrec + r] = prev[rc[r]];", GRADIENT),
    ("binomial-cost-slots-swapped", "fwi_oracle.c",
     "c[(size_t)(n - m) * (S + 1) + (s - 1)] + c[(size_t)m * (S + 1) + s]",
     "c[(size_t)(n - m) * (S + 1) + s] + c[(size_t)m * (S + 1) + (s - 1)]", GRADIENT),
    ("binomial-slot-not-consumed", "fwi_oracle.c", "oc_binom_gen(b, a + m_best, n - m_best, s - 1);",
     "oc_binom_gen(b, a + m_best, n - m_best, s);", GRADIENT),
    ("batch-stacked-at-grid-origin", "fwi_oracle.c",
     "            grad[(sh->x0 + i) + (long)g->nx * ((sh->y0 + j) + (long)g->ny * (sh->z0 + k))] +=",
     "            grad[i + (long)g->nx * ((sh->y0 + j) + (long)g->ny * (sh->z0 + k))] +=", BATCH),
    ("batch-model-window-at-grid-origin", "fwi_oracle.c",
     "              m[(sh->x0 + i) + (long)g->nx * ((sh->y0 + j) + (long)g->ny * (sh->z0 + k))];",
     "              m[i + (long)g->nx * ((sh->y0 + j) + (long)g->ny * (sh->z0 + k))];", BATCH),
    ("laplacian-missing-h2", "fwi_oracle.c", "double ih2 = 1.0 / (g->h * g->h);", "double ih2 = 1.0 / g->h;", STENCIL),
    ("laplacian-centre-weight", "fwi_oracle.c", "double acc = 3.0 * OC[0] * c;", "double acc = OC[0] * c;", STENCIL),
    ("source-doubled", "fwi_oracle.c", "Lbuf[cell[i]] += val[i];", "Lbuf[cell[i]] += 2.0 * val[i];", STENCIL),
    ("leapfrog-factor-two", "fwi_oracle.c", "out[i] = (2.0 * m[i] * idt2 * cur[i]", "out[i] = (m[i] * idt2 * cur[i]",
     STENCIL),
    ("damping-missing-in-a-plus", "fwi_oracle.c", "double ap = m[i] * idt2 + sig[i] / (2.0 * g->dt);",
     "double ap = m[i] * idt2;", STENCIL),
    ("sponge-depth-off-by-one", "fwi_oracle.c", "if (i < nbl) d = (nbl - i) * h;", "if (i < nbl) d = (nbl - i - 1) * h;",
     STENCIL),
    ("misfit-missing-half", "fwi_oracle.c", "phi += 0.5 * resid[i] * resid[i];", "phi += resid[i] * resid[i];",
     GRADIENT),
    ("residual-sign", "fwi_oracle.c", "resid[i] = dsim[i] - d_obs[i];", "resid[i] = d_obs[i] - dsim[i];", GRADIENT),
    ("codec-dequantise-exponent", "zfp_oracle.c", "ldexp((double)q[i], emax - ZO_S)", "ldexp((double)q[i], emax - ZO_S + 1)",
     CODEC),
    ("codec-half-truncates", "zfp_oracle.c", "return (int32_t)floor((double)a / 2.0);", "return a / 2;", CODEC),
    ("codec-no-plane-raise", "zfp_oracle.c", "if (p == 30 || p == 31) p = 32;", "if (p == 31) p = 32;", CODEC),
    ("codec-length-table-off-by-one", "zfp_oracle.c", "lengths[b] = (uint16_t)(bw.pos - before);",
     "lengths[b] = (uint16_t)(bw.pos - before + 1);", CODEC),
    ("codec-gather-x-y-swapped", "zfp_oracle.c",
     "      float v[64];\n      zo_gather(in, nx, ny, nz, &L, b, v);",
     "      float v[64], t[64];\n      zo_gather(in, nx, ny, nz, &L, b, t);\n"
     "      for (int q = 0; q < 64; q++) v[q] = t[((q >> 2) & 3) + 4 * (q & 3) + 16 * (q >> 4)];", CODEC),
    ("codec-guard-planes", "zfp_oracle.c", "#define ZO_G 11", "#define ZO_G 8", CODEC),
    ("codec-fraction-bits", "zfp_oracle.c", "#define ZO_S 25", "#define ZO_S 24", CODEC),
    ("codec-lifting-trend", "zfp_oracle.c", "  d0 = d0 - zo_half(D);\n  d1 = d1 - zo_half(D);\n  p[0] = S;",
     "  d1 = d1 - zo_half(D);\n  p[0] = S;", CODEC),
    ("codec-negabinary-mask", "zfp_oracle.c", "#define ZO_NBMASK 0xAAAAAAAAu", "#define ZO_NBMASK 0x55555555u", CODEC),
    ("codec-dropped-verbatim-bit", "zfp_oracle.c",
     "    for (int i = 0; i < n; i++)\n      if ((s = zo_put_bit(bw, (u[i] >> b) & 1u))) return s;",
     "    for (int i = 1; i < n; i++)\n      if ((s = zo_put_bit(bw, (u[i] >> b) & 1u))) return s;", CODEC),
]


def _build(tmp, mutation=None):
    """Copy the oracle sources into tmp, plant `mutation`, build liboracle.so there."""
    for f in ("fwi_oracle.c", "zfp_oracle.c", "oracle.h"):
        shutil.copy(os.path.join(ORACLE, f), tmp)
    if mutation:
        fname, old, new = mutation
        path = os.path.join(tmp, fname)
        src = open(path).read()
        assert src.count(old) == 1, f"mutation text not found exactly once in {fname}: {old!r}"
        open(path, "w").write(src.replace(old, new))
    lib = os.path.join(tmp, "liboracle.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wno-unknown-pragmas", "-o", lib,
                    os.path.join(tmp, "fwi_oracle.c"), os.path.join(tmp, "zfp_oracle.c"), "-lm"], check=True)
    return lib


def _pins(lib, test_file, stop_first=True, threads=None):
    env = dict(os.environ, ORACLE_LIBRARY=lib,
               OMP_NUM_THREADS=str(threads) if threads else os.environ.get("OMP_NUM_THREADS", "4"))
    cmd = [sys.executable, "-m", "pytest", test_file, "-q", "-m", "not gpu", "-p", "no:cacheprovider"]
    if stop_first:
        cmd.append("-x")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmutated_copy_passes_the_pins(tmp_path):
    lib = _build(str(tmp_path))
    for f in (STENCIL, GRADIENT, CODEC):
        r = _pins(lib, f, stop_first=False)
        assert r.returncode == 0, r.stdout[-2000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    """All mutations, several at a time (each in its own build and process)."""
    def run(mutant):
        mid, fname, old, new, pins = mutant
        d = tmp_path / mid
        d.mkdir()
        lib = _build(str(d), (fname, old, new))
        return mid, pins, _pins(lib, pins, threads=1)

    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(run, MUTANTS))
    missed = [f"{mid} ({pins}): exit {r.returncode}\n{r.stdout[-600:]}" for mid, pins, r in results
              if r.returncode != 1]
    assert not missed, "planted mistakes no pin caught:\n" + "\n".join(missed)
