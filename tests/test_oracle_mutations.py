"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/oracle.c`` (on the CPU),
builds it, and runs the pin suite against that copy: the suite must fail.
"""
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, text in oracle.c, replacement)
MUTATIONS = [
    ("rk4 third stage at h/2 (the printed listing)",
     "tmp[i] = y[i] + h * k3[i];", "tmp[i] = y[i] + (h / 2.0) * k3[i];"),
    ("rk4 weight of k3", "2.0 * k3[i] + k4[i]", "k3[i] + k4[i]"),
    ("rk4 update without h", "y[i] = y[i] + (h / 6.0) *", "y[i] = y[i] + (1.0 / 6.0) *"),
    ("traffic congestion term reads own cell",
     "s->w * (s->xbar - x[i + 1])", "s->w * (s->xbar - x[i])"),
    ("traffic inflow dropped", "double in = (i == 0) ? p[0] :", "double in = (i == 0) ? 0.0 :"),
    ("traffic last cell has no outflow",
     "if (i == s->n - 1) return min2(s->cap, s->v * x[i]);", "if (i == s->n - 1) return 0.0;"),
    ("ks second-derivative sign", "s->a1 = -s->g_2 * d2 + 4.0", "s->a1 = s->g_2 * d2 + 4.0"),
    ("ks a2 coefficient", "s->a2 = -s->g_4 * d4;", "s->a2 = -2.0 * s->g_4 * d4;"),
    ("ks advection direction", "double ux = (up1 - um1)", "double ux = (um1 - up1)"),
    ("ks decomposition min/max swapped", "(Da <= Db) ? min2(ea, eb) : max2(ea, eb)",
     "(Da <= Db) ? max2(ea, eb) : min2(ea, eb)"),
    ("ks decomposition neighbour transposed",
     "double Da = (x[ip1] - xh[im1])", "double Da = (xh[ip1] - x[im1])"),
    ("osc decomposition uses own x", "double z = xh[i];", "double z = x[i];"),
    ("osc cubic power", "s->kb * x[i] * x[i] * x[i]", "s->kb * x[i] * x[i]"),
    ("osc fixed end", "double xr = (i < m - 1) ? x[i + 1] : 0.0;\n        dy[i] = v[i];\n        dy[m + i] = -s->ka * x[i]",
     "double xr = (i < m - 1) ? x[i + 1] : x[i];\n        dy[i] = v[i];\n        dy[m + i] = -s->ka * x[i]"),
    ("linear decomposition sign split swapped",
     "else acc += posp(a) * x[j] + negp(a) * xh[j];", "else acc += negp(a) * x[j] + posp(a) * xh[j];"),
    ("traffic growth bound entries swapped", "if (i > 0) acc += s->v * r[i - 1];",
     "if (i > 0) acc += s->w * r[i - 1];"),
    ("traffic growth bound without input",
     "if (i < s->n - 1) acc += s->w * r[i + 1];\n        dr[i] = acc + ((i == 0) ? hp[0] : 0.0);",
     "if (i < s->n - 1) acc += s->w * r[i + 1];\n        dr[i] = acc;"),
    ("ks growth diagonal uses the infimum", "double Cii = max2(s->a0 - k * dmin, s->a0 - k * dmax);",
     "double Cii = min2(s->a0 - k * dmin, s->a0 - k * dmax);"),
    ("osc growth bound drops the radius", "double amax = fabs(cx[i]) + rx[i];", "double amax = fabs(cx[i]);"),
    ("linear growth bound keeps the sign", "acc += ((j == i) ? a : fabs(a)) * r[j];", "acc += a * r[j];"),
    ("mm inputs swapped", "c.s = s; c.p = wlo; c.ph = whi;", "c.s = s; c.p = whi; c.ph = wlo;"),
    ("cgb center is the lower corner", "z[i] = (xlo[i] + xhi[i]) / 2.0;", "z[i] = xlo[i];"),
    ("mc samples the input stream for x0", "orc_uniform(seed, j, i, 0u);", "orc_uniform(seed, j, i, 1u);"),
    ("mc inputs not sampled", "p[k] = wlo[k] + (whi[k] - wlo[k]) * orc_uniform(seed, j, k, 1u);",
     "p[k] = wlo[k];"),
    ("philox multiplier", "0xD2511F53u", "0xD2511F55u"),
    ("philox key schedule", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;"),
    ("uniform uses 52 bits", "(bits >> 11) * 0x1.0p-53", "(bits >> 12) * 0x1.0p-52"),
    ("heat open face ignored", "else if (s->open) acc += 0.0 - u[i];", "else if (s->open) acc += 0.0;"),
    ("heat y neighbour index", "if (y < l - 1) acc += u[i + l] - u[i];", "if (y < l - 1) acc += u[i + 1] - u[i];"),
    ("heat coefficient", "s->kh = alpha / (dx * dx);", "s->kh = alpha / dx;"),    ('quad north acceleration sign', 'dy[3] = a * (-(cf * st * cp) - sf * sp);', 'dy[3] = a * (-(cf * st * cp) + sf * sp);'),
    ('quad east acceleration uses cos psi', 'dy[4] = a * (-(cf * st * sp) + sf * cp);', 'dy[4] = a * (-(cf * st * cp) + sf * cp);'),
    ('quad vertical acceleration drops cos theta', 'dy[5] = s->qg - a * (cf * ct);', 'dy[5] = s->qg - a * cf;'),
    ('quad inertia swapped', '        dy[10] = tau[1] / s->Jy;\n        dy[11] = tau[2] / s->Jz;\n    }\n}\n\nstatic void f_sys', '        dy[10] = tau[1] / s->Jx;\n        dy[11] = tau[2] / s->Jz;\n    }\n}\n\nstatic void f_sys'),
    ('quad agent input stride', 'const double *y = x + 12 * k, *tau = p + 3 * k;', 'const double *y = x + 12 * k, *tau = p + 2 * k;'),
    ('quad interval sin misses its maximum', 'r.hi = holds_point(a.lo, a.hi, ORC_HALF_PI) ? 1.0 : max2(s0, s1);', 'r.hi = max2(s0, s1);'),
    ('quad extremum test takes the point one period before a',
     'return p <= b;', 'return p - ORC_TWO_PI <= b;'),
    ('quad extremum test compares with the wrong end', 'return p <= b;', 'return p <= a;'),
    ('quad interval cos minimum point', 'r.lo = holds_point(a.lo, a.hi, ORC_PI) ? -1.0 : min2(c0, c1);', 'r.lo = holds_point(a.lo, a.hi, ORC_HALF_PI) ? -1.0 : min2(c0, c1);'),
    ('quad interval product drops a corner', 'ival r = {min2(min2(p1, p2), min2(p3, p4)), max2(max2(p1, p2), max2(p3, p4))};', 'ival r = {min2(p1, p4), max2(p1, p4)};'),
    ('quad decomposition orientation', 'dy[3] = lower ? an.lo : an.hi;', 'dy[3] = lower ? an.hi : an.lo;'),
    ('quad growth drops the psi column', 'd[3] = n_f * rr[6] + n_t * rr[7] + n_p * rr[8];', 'd[3] = n_f * rr[6] + n_t * rr[7];'),
    ('quad growth derivative sign', 'double n_f = a * iv_mag(iv_add(iv_mul(iv_mul(sf, st), cp), iv_neg(iv_mul(cf, sp))));', 'double n_f = a * iv_mag(iv_add(iv_mul(iv_mul(sf, st), cp), iv_mul(cf, sp)));'),
    ('quad growth input not scaled by inertia', 'd[9] = hw[0] / s->Jx;', 'd[9] = hw[0];'),
    ('quad growth box from the center only', 'ival F = {cc[6] - rr[6], cc[6] + rr[6]}', 'ival F = {cc[6], cc[6]}'),
    ('traffic local: free flow certain ignores congestion', 'return j == s->n - 1 || f < s->w * (s->xbar - hi[j + 1]);', 'return 1;'),
    ('traffic local: congestion possible ignores capacity', 'return q <= s->cap && q <= s->v * hi[j];', 'return q <= s->v * hi[j];'),
    ('traffic local: congested-inflow diagonal dropped', 'if (i > 0 && tr_cong_certain(s, lo, i - 1)) cd -= s->w;', ''),
    ('traffic local: free flow possible tested at the upper corner', 'double cl = (i > 0 && tr_ff_possible(s, lo, i - 1)) ? s->v : 0.0;', 'double cl = (i > 0 && tr_ff_possible(s, hi, i - 1)) ? s->v : 0.0;'),
    ('traffic local: superdiagonal keeps w', 'double cr = tr_cong_possible(s, hi, i) ? s->w : 0.0;', 'double cr = s->w;'),
    ('sound: flux difference rounded up for the lower end', 'kl[i] = add_dn(inl, -outu);', 'kl[i] = add_up(inl, -outu);'),
    ('sound: congestion term from the wrong end', '*fl = min2(s->cap, min2(vl, mul_dn(s->w, add_dn(s->xbar, -yu[i + 1]))));', '*fl = min2(s->cap, min2(vl, mul_dn(s->w, add_dn(s->xbar, -yl[i + 1]))));'),
    ('sound: h/6 bound ignores the sign', '*rl = mul_dn(ql >= 0.0 ? cl : cu, ql);', '*rl = mul_dn(cl, ql);'),
    ('sound: radius product rounded down', 'if (i > 0) acc = add_up(acc, mul_up(s->v, r[i - 1]));', 'if (i > 0) acc = add_up(acc, mul_dn(s->v, r[i - 1]));'),
    ('sound: downward sum rounds to nearest', '    double s = a + b, bb = s - a, e = (a - (s - bb)) + (b - bb);\n    return e < 0.0 ? nextafter(s, -INFINITY) : s;', '    double s = a + b;\n    return s;'),
    ('sound: center rounded to nearest', 'cl[i] = 0.5 * add_dn(xlo[i], xhi[i]);', 'cl[i] = 0.5 * (xlo[i] + xhi[i]);'),
]


def _run_mutation(mut, workdir):
    """Build the mutated oracle and run the pins against it; True when they fail."""
    name, old, new = mut
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    os.makedirs(workdir, exist_ok=True)
    mutated = os.path.join(workdir, "oracle.c")
    with open(mutated, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(workdir, "liboracle_mut.so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared",
                           "-o", lib, mutated, "-lm"])
    env = dict(os.environ, REACH_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(HERE, "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode != 0, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Every mutation run once, concurrently (each is a compiler call and a
    pytest subprocess, so threads only wait on them)."""
    from concurrent.futures import ThreadPoolExecutor
    base = tmp_path_factory.mktemp("mutations")
    workers = max(1, min(len(MUTATIONS), os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        futs = {m[0]: ex.submit(_run_mutation, m, str(base / f"m{k}")) for k, m in enumerate(MUTATIONS)}
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.parametrize("mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_mutation(mut, outcomes):
    caught, log = outcomes[mut[0]]
    assert caught, f"pins did not catch: {mut[0]}\n{log}"
