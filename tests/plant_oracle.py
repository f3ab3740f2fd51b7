"""Planted-mistake check of the oracle's pins (run by hand, not collected by pytest).

Each entry plants one plausible mistake (a dropped term or factor, a wrong sign, index or argument
order) into a copy of ``oracle/``, runs the CPU oracle tests against the copy and reports whether a
pin fails.  A mistake that no pin catches is listed in EQUIVALENT with the reason (an equivalent
change, or a change of a documented reading) or is a gap to close with a new pin.

    python tests/plant_oracle.py [--workdir DIR] [--only NAME_PREFIX]

Each run copies oracle/, synthetic/ and tests/ into DIR (a fresh temporary folder by default) and
takes about a minute per uncaught plant (the whole CPU oracle suite), seconds per caught one.
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = ["tests/test_oracle_harmonics.py", "tests/test_oracle_power.py", "tests/test_oracle_mesh.py",
         "tests/test_oracle_bispec.py", "tests/test_oracle_sugiyama.py", "tests/test_oracle_adjoint.py",
         "tests/test_golden.py"]

# (name, file, text, replacement, occurrences)
PLANTS = [
    ("P1 N0 with alpha for alpha^2", "oracle/power.py",
     "n0 = (_fsum(wg**2) + alpha**2 * _fsum(wr**2)) / i22", "n0 = (_fsum(wg**2) + alpha * _fsum(wr**2)) / i22", 1),
    ("P2 I22 without alpha", "oracle/power.py", "i22 = alpha * _fsum(nr * wr**2)", "i22 = _fsum(nr * wr**2)", 1),
    ("P3 randoms added, not subtracted", "oracle/power.py",
     'coef = -scalars["alpha"] if weight_power == 1', 'coef = scalars["alpha"] if weight_power == 1', 1),
    ("P4 interlacing phase conjugated", "oracle/power.py",
     "s = 0.5 * (parts[0] + M.interlace_phase(n) * parts[1])",
     "s = 0.5 * (parts[0] + np.conj(M.interlace_phase(n)) * parts[1])", 1),
    ("P5 m > 0 terms not doubled", "oracle/power.py",
     "acc = acc + 2.0 * np.conj(H.ylm(ell, m, kh))", "acc = acc + 1.0 * np.conj(H.ylm(ell, m, kh))", 1),
    ("P6 Hand+17 Y_lm not conjugated", "oracle/power.py",
     "acc += np.conj(H.ylm(ell, m, kh)) * ylm_transform", "acc += H.ylm(ell, m, kh) * ylm_transform", 1),
    ("P8 inversion index off by one", "oracle/power.py",
     "np.roll(np.flip(g, axis=(0, 1, 2)), 1, axis=(0, 1, 2))", "np.flip(g, axis=(0, 1, 2))", 1),
    ("P9a shot noise from every l", "oracle/power.py", "- (n0 if ell == 0 else 0.0))", "- n0)", 2),
    ("P9b (l+1) for (2l+1)", "oracle/power.py", "(2 * ell + 1) / i22 * mean", "(ell + 1) / i22 * mean", 3),
    ("P10 N_ll' denominator", "oracle/power.py", "return (2 * (ell + ellp) + 1) * n0 / (2 * ell + 1)",
     "return (2 * (ell + ellp) + 1) * n0 / (2 * ell + 3)", 1),
    ("P11 a P_lb coefficient", "oracle/power.py", "(2, 2): Fraction(35, 18)", "(2, 2): Fraction(35, 17)", 1),
    ("P12 odd l from the real part", "oracle/power.py", "return np.imag(z) if ell % 2 else np.real(z)",
     "return np.real(z)", 1),
    ("P13 P_ll' not conjugated", "oracle/power.py", "v = np.real(ff[a] * np.conj(ff[c]))",
     "v = np.real(ff[a] * ff[c])", 1),
    ("P14 S with +alpha^3", "oracle/power.py", "s3 = _fsum(wg**3) - alpha**3 * _fsum(wr**3)",
     "s3 = _fsum(wg**3) + alpha**3 * _fsum(wr**3)", 1),
    ("P15 I33 with alpha^2", "oracle/power.py", "i33 = alpha * _fsum(nr**2 * wr**3)",
     "i33 = alpha**2 * _fsum(nr**2 * wr**3)", 1),
    ("P16 S with alpha^2", "oracle/power.py", "s3 = _fsum(wg**3) - alpha**3 * _fsum(wr**3)",
     "s3 = _fsum(wg**3) - alpha**2 * _fsum(wr**3)", 1),
    ("P17 periodic I33 over V", "oracle/power.py", "i33 = wsum**3 / vol**2", "i33 = wsum**3 / vol", 1),
]
PLANTS += [
    ("H1 Y_lm norm inverted", "oracle/harmonics.py", "factorial(ell - am) / factorial(ell + am))",
     "factorial(ell + am) / factorial(ell - am))", 1),
    ("H2 Y_l^-m without (-1)^m", "oracle/harmonics.py", "return (-1.0) ** am * np.conj(pos)", "return np.conj(pos)", 1),
    ("H3 3j phase", "oracle/harmonics.py", "sign = -1.0 if (j1 - j2 - m3) % 2 else 1.0",
     "sign = -1.0 if (j1 - j2 + m1) % 2 else 1.0", 1),
    ("H4 3j triangle factor", "oracle/harmonics.py", "f(j1 + j2 + j3 + 1))", "f(j1 + j2 + j3))", 1),
    ("M1 phase b shifted the wrong way", "oracle/mesh.py", "* inv_h + shift", "* inv_h - shift", 1),
    ("K1 TSC centre weight", "oracle/mesh.py", "(0, 0.75 - d * d)", "(0, 0.75 - 0.5 * d * d)", 1),
    ("B2 (l+1) for (2l+1) in B_l", "oracle/bispec.py", "B[ell] = np.where(nt > 0, (2 * ell + 1) * s / (i33",
     "B[ell] = np.where(nt > 0, (ell + 1) * s / (i33", 2),
    ("B3 N_T scale", "oracle/bispec.py", "for i, j, k in tri]) / n**3", "for i, j, k in tri]) / n**2", 6),
    ("B4 compressed normalisation", "oracle/bispec.py",
     "hnorm = H.wigner3j(ell, 0, ell, 0, 0, 0) * (2 * ell + 1) ** 2",
     "hnorm = H.wigner3j(ell, 0, ell, 0, 0, 0) * (2 * ell + 1)", 1),
    ("B5 odd shells from the real part", "oracle/bispec.py",
     "a[ib] = np.imag(np.fft.ifftn(np.where(b == ib, Xl[ell], 0.0))) * n**3",
     "a[ib] = np.real(np.fft.ifftn(np.where(b == ib, Xl[ell], 0.0))) * n**3", 1),
    ("S1 FFT-method shot -S for -2S", "oracle/shot.py",
     'tot = np.real(t["t23"] + t["t12"] + t["t13"]) - 2.0 * s3 * t["ntl"]',
     'tot = np.real(t["t23"] + t["t12"] + t["t13"]) - 1.0 * s3 * t["ntl"]', 1),
    ("S2 compressed FFT-method shot -S", "oracle/shot.py", "np.real(ta + tb + tc - 2.0 * s3 * td)",
     "np.real(ta + tb + tc - s3 * td)", 1),
    ("S3 analytic shot cosines swapped", "oracle/shot.py",
     "v += float(H.legendre(ell, c12)) * hl[j] + float(H.legendre(ell, c13)) * hl[k]",
     "v += float(H.legendre(ell, c13)) * hl[j] + float(H.legendre(ell, c12)) * hl[k]", 1),
    ("S4 analytic shot g_l argument", "oracle/shot.py", "v += sgn * H.g_ell(ell, c[i] / c[j]) * hl[i]",
     "v += sgn * H.g_ell(ell, c[j] / c[i]) * hl[i]", 1),
    ("G1 TripoSH (2L+1) dropped", "oracle/sugiyama.py", "* (2 * l1 + 1) * (2 * l2 + 1) * (2 * L + 1)",
     "* (2 * l1 + 1) * (2 * l2 + 1)", 5),
    ("G2 TripoSH 3j m1, m2 swapped", "oracle/sugiyama.py", "w = H.wigner3j(l1, l2, L, m1, m2, Mm)",
     "w = H.wigner3j(l1, l2, L, m2, m1, Mm)", 4),
    ("G3 Lemma 1 sign", "oracle/sugiyama.py", "s += (-1.0) ** n * float(", "s += float(", 1),
    ("G4 paired half-sum weight", "oracle/sugiyama.py", "eta = 1.0 if (m1, m2, Mm) == (0, 0, 0) else 2.0",
     "eta = 1.0", 1),
    ("G5 TripoSH shot k1 term on k2", "oracle/sugiyama.py", "v += (2 * L + 1) / i33 * Hk[L][i]",
     "v += (2 * L + 1) / i33 * Hk[L][j]", 1),
    ("A1 adjoint factor 2 dropped", "oracle/adjoint.py", "Y = 2.0 * K * X / M.window(n, assign)",
     "Y = K * X / M.window(n, assign)", 1),
    ("HS1 half spectrum m > 0 not doubled", "oracle/power.py",
     "c = 4.0 * pi / (2 * ell + 1) * (1.0 if m == 0 else 2.0)", "c = 4.0 * pi / (2 * ell + 1) * 1.0", 1),
    ("HS2 half spectrum imaginary part sign", "oracle/power.py",
     "term += c * np.imag(yk) * self._rfft(mesh * np.imag(y))",
     "term -= c * np.imag(yk) * self._rfft(mesh * np.imag(y))", 1),
    ("HS3 half spectrum pair weight", "oracle/power.py", "wgt = (np.where(iz == 0, 1.0, 2.0) * ok).ravel()",
     "wgt = (np.where(iz == 0, 2.0, 2.0) * ok).ravel()", 1),
    ("HS4 half spectrum Nyquist plane kept", "oracle/power.py", "& (iz != n // 2)", "", 1),
    ("HS5 half spectrum interlacing phase", "oracle/power.py", "ph = np.exp(1j * a * (ix + iy + iz))",
     "ph = np.exp(-1j * a * (ix + iy + iz))", 1),
    ("X1 cross I22 of tracer A only", "oracle/power.py", 'i22 = np.sqrt(sa["I22"] * sb["I22"])', 'i22 = sa["I22"]', 1),
    ("X2 cross tracers swapped", "oracle/power.py", "_part(ell, fa[0] * np.conj(fb[ell]))",
     "_part(ell, fb[0] * np.conj(fa[ell]))", 1),
    ("SV1 survey self-term moments with alpha^2", "oracle/shot.py", "v -= alpha ** 3 * np.sum(",
     "v -= alpha ** 2 * np.sum(", 1),
    ("TS1 TripoSH G field not conjugated", "oracle/sugiyama.py",
     "lambda sh, L=L, Mm=Mm: np.conj(H.ylm_racah(L, Mm, P._xhat_dirs(spec, sh))))",
     "lambda sh, L=L, Mm=Mm: H.ylm_racah(L, Mm, P._xhat_dirs(spec, sh)))", 1),
    ("TS2 TripoSH shell weight not conjugated", "oracle/sugiyama.py",
     "w = np.conj(H.ylm_racah(ell, m, P._khat(spec))) * X0", "w = H.ylm_racah(ell, m, P._khat(spec)) * X0", 1),
    ("AD2 bispectrum adjoint 3 -> 2", "oracle/adjoint.py", "c = 3.0 * dldb[k] / (i33 * nt)",
     "c = 2.0 * dldb[k] / (i33 * nt)", 1),
    ("L1 global line of sight not normalised", "oracle/bispec.py",
     "    d = d / np.linalg.norm(d)\n    kk = np.sqrt(kx * kx + ky * ky + kz * kz)",
     "    kk = np.sqrt(kx * kx + ky * ky + kz * kz)", 1),
]

# Uncaught, and why: the first two give the same result for every input the oracle takes; the
# third changes only a reading that no printed value fixes; the fourth is a limit of the pins.
EQUIVALENT = [
    ("survey self term S_l not conjugated", "oracle/shot.py",
     "the survey shot noise is formed for l = 0 (real Y_00 and C_00) and l = 2, where every bin is a "
     "union of lattice shells invariant under the cube's symmetries, so <Y_2m>_k = 0 and S_2 = 0"),
    ("survey Q_l built as H_l (line of sight on the wrong leg)", "oracle/shot.py",
     "NOT PINNED beyond the distant-observer limit, where Q_l = H_l; without randoms N = w F and "
     "Q_l = H_l exactly, so no few-object identity separates them, only a statistical test with "
     "randoms near the observer"),
    ("(-1)^l dropped from the space inversion", "oracle/power.py",
     "F_l from G_l is formed only for the even l = 2, 4 of the two-index spectra, where (-1)^l = 1"),
    ("strict bin-centre closure c_k < c_i + c_j", "oracle/bispec.py",
     "the rules differ only when a bin centre equals the sum of two others, which needs kmin = dk/2 "
     "(mod dk): never for the bench workloads' bins (from 0 and from dk; 805 triangles at 19 bins is "
     "pinned), and the tests with bins from k_f/2 check identities that hold for any triangle set. "
     "Whether the flat triangle c_k = c_i + c_j counts is a reading of Sec. 2.2's closed triangles"),
]


def run(workdir, name, fn, old, new, count):
    d = os.path.join(workdir, "".join(ch if ch.isalnum() else "_" for ch in name))
    if os.path.isdir(d):
        shutil.rmtree(d)
    os.makedirs(d)
    for sub in ("oracle", "synthetic", "tests"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                        ignore=shutil.ignore_patterns("__pycache__"))
    path = os.path.join(d, fn)
    with open(path) as f:
        src = f.read()
    if src.count(old) != count:
        shutil.rmtree(d)
        return "PATTERN COUNT %d (expected %d): update the plant" % (src.count(old), count)
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "-m", "not gpu and not slow"] + TESTS, cwd=d, capture_output=True, text=True)
    shutil.rmtree(d)
    failed = [ln for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
    if r.returncode == 0:
        return "MISSED"
    return "caught by " + (failed[0].split(" ")[1] if failed else "an error: " + r.stdout[-200:])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workdir", default=None)
    ap.add_argument("--only", default="")
    args = ap.parse_args()
    workdir = args.workdir or tempfile.mkdtemp(prefix="plant_oracle_")
    os.makedirs(workdir, exist_ok=True)
    missed = 0
    for name, fn, old, new, count in PLANTS:
        if not name.startswith(args.only):
            continue
        res = run(workdir, name, fn, old, new, count)
        missed += not res.startswith("caught")
        print("%-40s %s" % (name, res), flush=True)
    for name, fn, why in EQUIVALENT:
        print("%-40s equivalent (%s): %s" % (name, fn, why))
    return 1 if missed else 0


if __name__ == "__main__":
    sys.exit(main())
