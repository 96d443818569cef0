"""Derive the polynomial coefficients of the FP64 sin/cos helper (exa_fp64_sincos.inc).

On the reduced interval |r| <= pi/4, with z = r^2:

    sin r ~ r + r^3 * S(z),          S of degree 5 in z (r^3 ... r^13)
    cos r ~ 1 - z/2 + z^2 * C(z),     C of degree 5 in z (r^4 ... r^14)

S and C minimise the largest RELATIVE error of sin r and cos r over z in [0, (pi/4)^2].  They are
found with the Remez exchange algorithm (E. Ya. Remez, 1934) for a weighted polynomial fit: a
degree-n polynomial p that minimises max |w(z) (p(z) - g(z))| equioscillates at n + 2 points, so
each iteration solves the linear system of that equioscillation on the current reference points and
moves the reference to the extrema of the new error curve.  Here

    sin:  g(z) = (sin r - r) / r^3,        w(z) = z r / sin r      (error of sin r relative to sin r)
    cos:  g(z) = (cos r - 1 + z/2) / z^2,  w(z) = z^2 / cos r

All arithmetic runs in 60-digit mpmath.  The coefficients are then rounded to the nearest double and
the relative error of the rounded polynomials is measured on a dense grid.  Running the script prints
the coefficients as C hex-float literals together with those error bounds; `check()` is what the
CPU tests call.
"""
import mpmath as mp

mp.mp.dps = 60
PI4 = mp.pi / 4
ZMAX = PI4 * PI4
DEG = 5


def _g_sin(z):
    r = mp.sqrt(z)
    return (mp.sin(r) - r) / (r * z)


def _w_sin(z):
    r = mp.sqrt(z)
    return z * r / mp.sin(r)


def _g_cos(z):
    r = mp.sqrt(z)
    return (mp.cos(r) - 1 + z / 2) / (z * z)


def _w_cos(z):
    return z * z / mp.cos(mp.sqrt(z))


def _poly(c, z):
    acc = mp.mpf(0)
    for a in reversed(c):
        acc = acc * z + a
    return acc


def _err(c, g, w, z):
    return w(z) * (_poly(c, z) - g(z))


def _extrema(c, g, w, lo, hi, npts=3000):
    """Alternating extrema of the weighted error on a dense grid (interior local extrema, then the
    right end point), each refined by golden-section search on |e|."""
    zs = [lo + (hi - lo) * mp.mpf(i) / npts for i in range(npts + 1)]
    es = [_err(c, g, w, z) for z in zs]
    idx = [i for i in range(1, npts) if abs(es[i]) >= abs(es[i - 1]) and abs(es[i]) >= abs(es[i + 1])]
    idx.append(npts)
    pts = []
    for i in idx:
        a, b = zs[max(i - 1, 0)], zs[min(i + 1, npts)]
        if i == npts:
            pts.append(zs[i])
            continue
        phi = (mp.sqrt(5) - 1) / 2
        x1, x2 = b - phi * (b - a), a + phi * (b - a)
        f1, f2 = abs(_err(c, g, w, x1)), abs(_err(c, g, w, x2))
        for _ in range(60):
            if f1 > f2:
                b, x2, f2 = x2, x1, f1
                x1 = b - phi * (b - a)
                f1 = abs(_err(c, g, w, x1))
            else:
                a, x1, f1 = x1, x2, f2
                x2 = a + phi * (b - a)
                f2 = abs(_err(c, g, w, x2))
        pts.append((a + b) / 2)
    # keep an alternating sequence, the larger of neighbours with equal sign
    out = []
    for z in pts:
        e = _err(c, g, w, z)
        if out and mp.sign(out[-1][1]) == mp.sign(e):
            if abs(e) > abs(out[-1][1]):
                out[-1] = (z, e)
        else:
            out.append((z, e))
    return out


def remez(g, w, n=DEG, lo=None, hi=ZMAX, iters=30):
    lo = hi * mp.mpf("1e-8") if lo is None else lo
    # initial reference: Chebyshev extrema on [lo, hi]
    ref = [lo + (hi - lo) * (1 - mp.cos(mp.pi * i / (n + 1))) / 2 for i in range(n + 2)]
    c = None
    for _ in range(iters):
        A = mp.matrix(n + 2, n + 2)
        rhs = mp.matrix(n + 2, 1)
        for i, z in enumerate(ref):
            for j in range(n + 1):
                A[i, j] = z ** j
            A[i, n + 1] = (-1) ** i / w(z)
            rhs[i] = g(z)
        sol = mp.lu_solve(A, rhs)
        c = [sol[j] for j in range(n + 1)]
        ext = _extrema(c, g, w, lo, hi)
        if len(ext) < n + 2:
            break
        # the n + 2 consecutive extrema holding the largest one
        k = max(range(len(ext)), key=lambda i: abs(ext[i][1]))
        s = min(max(k - (n + 1) // 2, 0), len(ext) - (n + 2))
        new = [z for z, _ in ext[s:s + n + 2]]
        big = max(abs(e) for _, e in ext)
        small = min(abs(e) for _, e in ext[s:s + n + 2])
        ref = new
        if big / small - 1 < mp.mpf("1e-6"):
            break
    return c


def to_double(c):
    return [float(a) for a in c]


def rel_error_of_rounded(kind, cd, npts=4000):
    """Largest relative error, in exact arithmetic, of the polynomial with double coefficients."""
    worst = mp.mpf(0)
    for i in range(1, npts + 1):
        r = PI4 * mp.mpf(i) / npts
        z = r * r
        p = _poly([mp.mpf(a) for a in cd], z)
        if kind == "sin":
            approx, exact = r + r * z * p, mp.sin(r)
        else:
            approx, exact = 1 - z / 2 + z * z * p, mp.cos(r)
        worst = max(worst, abs(approx / exact - 1))
    return worst


def derive():
    s = to_double(remez(_g_sin, _w_sin))
    c = to_double(remez(_g_cos, _w_cos))
    return s, c


def check():
    """(sin coefficients, cos coefficients, sin bound, cos bound) as the script derives them now."""
    s, c = derive()
    return s, c, float(rel_error_of_rounded("sin", s)), float(rel_error_of_rounded("cos", c))


if __name__ == "__main__":
    s, c, es, ec = check()
    print("sin: S(z), lowest power first; largest relative error", es)
    for a in s:
        print("  ", a.hex())
    print("cos: C(z), lowest power first; largest relative error", ec)
    for a in c:
        print("  ", a.hex())
