"""Host model of the pair arithmetic of the refinement on FP32 pairs: the
error-free transformations (Knuth's two-sum, the product error by FMA) and the
heat residual formed from neighbour differences, evaluated in IEEE binary32
with numpy and compared with exact rational arithmetic.  This pins the error
bound the pair form relies on, independently of the GPU: the residual of the
represented values is lost below about
2^-48 (|x_j| + sum_i c_i (2 |x_j| + |x_m| + |x_p|)), the FP64 residual's
bound with 2^-48 in place of 2^-53 (the lo parts of the neighbour
differences are combined in FP32; the hi parts and products are exact).

FMA is modelled as fl32(a b + c) with a b exact in binary64 (two 24-bit
significands); for the product error fl32(a b - fl32(a b)) that is exact, as
the hardware FMA is."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bv = f32(s - a)
    e = f32(f32(a - f32(s - bv)) + f32(b - bv))
    return s, e


def fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def split(v):
    hi = f32(v)
    # truncation of the kernel vs rounding here: either leaves |lo| <= ulp(hi)
    lo = f32(np.float64(v) - np.float64(hi))
    return hi, lo


def exact(p):
    return Fraction(float(p[0])) + Fraction(float(p[1]))


def pair_heat_residual(x, b, j, nb, c):
    """The kernel's operation order for one node: x, b lists of (hi, lo);
    nb[i] = (m, p) neighbour indices or None; c[i] = (hi, lo) of dt / h_i^2."""
    xj, bj = x[j], b[j]
    s, comp = two_sum(bj[0], f32(-xj[0]))
    comp = f32(comp + f32(bj[1] - xj[1]))
    for i, (m, p) in enumerate(nb):
        xm = x[m] if m is not None else (f32(0), f32(0))
        xq = x[p] if p is not None else (f32(0), f32(0))
        a1, e1 = two_sum(xj[0], f32(-xm[0]))
        a2, e2 = two_sum(xj[0], f32(-xq[0]))
        t, e3 = two_sum(a1, a2)
        tl = f32(f32(f32(e1 + e2) + e3) + f32(f32(fma(f32(2), xj[1], f32(-xm[1]))) - xq[1]))
        ch, cl = c[i]
        pr = f32(ch * t)
        q = f32(fma(ch, t, f32(-pr)) + fma(ch, tl, f32(cl * t)))
        s, e4 = two_sum(s, f32(-pr))
        comp = f32(comp + f32(e4 - q))
    return f32(s + comp)


def test_two_sum_and_product_error_are_exact():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        a, b = f32(rng.normal() * 10.0 ** rng.integers(-8, 8)), f32(rng.normal() * 10.0 ** rng.integers(-8, 8))
        s, e = two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))
        p = f32(a * b)
        ep = fma(a, b, f32(-p))
        assert Fraction(float(p)) + Fraction(float(ep)) == Fraction(float(a)) * Fraction(float(b))


def test_split_keeps_48_bits():
    rng = np.random.default_rng(2)
    for _ in range(2000):
        v = rng.normal() * 10.0 ** rng.integers(-20, 20)
        hi, lo = split(v)
        assert abs(exact((hi, lo)) - Fraction(v)) <= abs(Fraction(v)) * Fraction(1, 2 ** 47)


def test_pair_heat_residual_floor():
    """1-D and 2-D heat stencils with dt / h^2 from 0.01 to 400, on smooth and
    random states, near the solution of the step (where b - A x cancels to
    the representation error) and away from it: the pair residual equals the
    exact residual of the represented values up to
    4 x 2^-48 (|x_j| + sum_i c_i (2 |x_j| + |x_m| + |x_p|)) plus one FP32
    rounding of the result."""
    rng = np.random.default_rng(3)
    worst = 0.0
    for trial in range(300):
        d = 1 + trial % 2
        n = 9
        c_val = [10.0 ** rng.uniform(-2, 2.6) for _ in range(d)]  # dt / h^2 up to 400
        c = [split(v) for v in c_val]
        shape = (n,) * d
        N = int(np.prod(shape))
        smooth = trial % 3 != 0
        grid = np.indices(shape).reshape(d, -1).T
        if smooth:
            base = np.prod(np.sin(np.pi * (grid + 1) / (n + 1)), axis=1)
        else:
            base = rng.normal(size=N)
        strides = [int(np.prod(shape[i + 1:])) for i in range(d)]
        bv = base
        if trial % 2 == 0:
            # near the solution of (I + dt L) x = b, where b - A x cancels to
            # the representation error: the floor decides
            A = np.eye(N)
            for jj in range(N):
                for i in range(d):
                    A[jj, jj] += 2 * c_val[i]
                    if grid[jj][i] > 0:
                        A[jj, jj - strides[i]] -= c_val[i]
                    if grid[jj][i] < n - 1:
                        A[jj, jj + strides[i]] -= c_val[i]
            xv = np.linalg.solve(A, bv)
        else:
            xv = base * (1.0 + 1e-3 * rng.normal(size=N))
        x = [split(v) for v in xv]
        b = [split(v) for v in bv]
        for j in range(N):
            coords = grid[j]
            nb = []
            for i in range(d):
                m = j - strides[i] if coords[i] > 0 else None
                p = j + strides[i] if coords[i] < n - 1 else None
                nb.append((m, p))
            r = pair_heat_residual(x, b, j, nb, c)
            xj = exact(x[j])
            ex = exact(b[j]) - xj
            scale = abs(xj)
            for i, (m, p) in enumerate(nb):
                xm = exact(x[m]) if m is not None else Fraction(0)
                xp = exact(x[p]) if p is not None else Fraction(0)
                ex -= exact(c[i]) * (2 * xj - xm - xp)
                scale += exact(c[i]) * (2 * abs(xj) + abs(xm) + abs(xp))
            err = abs(Fraction(float(r)) - ex)
            bound = 4 * scale / 2 ** 48 + abs(ex) / 2 ** 23
            assert err <= bound, (trial, j, float(err), float(bound))
            if scale > 0:
                worst = max(worst, float((err - abs(ex) / 2 ** 23) / scale))
    # the bound is not loose by orders of magnitude: the model reaches it
    assert 2 ** -52 < worst <= 4 / 2 ** 48


def pair_tab_residual(x, b, j, nb, cf):
    """The kernel's operation order for the variable-coefficient operator:
    nb[k] = neighbour index or None for k = 2 i (towards -e_i) and 2 i + 1;
    cf[k] = (hi, lo) of the face coefficient dt a / h_i^2."""
    xj, bj = x[j], b[j]
    s, comp = two_sum(bj[0], f32(-xj[0]))
    comp = f32(comp + f32(bj[1] - xj[1]))
    for k, n in enumerate(nb):
        xn = x[n] if n is not None else (f32(0), f32(0))
        dh, e1 = two_sum(xj[0], f32(-xn[0]))
        dl = f32(e1 + f32(xj[1] - xn[1]))
        ch, cl = cf[k]
        pr = f32(ch * dh)
        q = f32(fma(ch, dh, f32(-pr)) + fma(ch, dl, f32(cl * dh)))
        s, e2 = two_sum(s, f32(-pr))
        comp = f32(comp + f32(e2 - q))
    return f32(s + comp)


def test_pair_tab_residual_floor():
    """Variable coefficient (face coefficients from a = 1 + A sin cos, dt /
    h^2 up to 400), near the solution of the step and away from it: the same
    bound as the heat form, 4 x 2^-48 (|x_j| + sum_faces c (|x_j| + |x_n|))
    plus one FP32 rounding."""
    rng = np.random.default_rng(4)
    worst = 0.0
    for trial in range(200):
        d = 1 + trial % 2
        n = 8
        shape = (n,) * d
        N = int(np.prod(shape))
        grid = np.indices(shape).reshape(d, -1).T
        strides = [int(np.prod(shape[i + 1:])) for i in range(d)]
        cs = [10.0 ** rng.uniform(-2, 2.6) for _ in range(d)]
        # per node and face: c = dt a(face) / h^2 with a smooth positive a
        cval = np.empty((N, 2 * d))
        for j in range(N):
            for i in range(d):
                for side in (0, 1):
                    xf = (grid[j][i] + 1 + (side - 0.5)) / (n + 1)
                    cval[j, 2 * i + side] = cs[i] * (1.0 + 0.5 * np.sin(2 * np.pi * xf))
        nbs = []
        for j in range(N):
            nb = []
            for i in range(d):
                nb.append(j - strides[i] if grid[j][i] > 0 else None)
                nb.append(j + strides[i] if grid[j][i] < n - 1 else None)
            nbs.append(nb)
        bv = rng.normal(size=N) if trial % 3 == 0 else np.prod(np.sin(np.pi * (grid + 1) / (n + 1)), axis=1)
        if trial % 2 == 0:
            A = np.eye(N)
            for j in range(N):
                for k, nn in enumerate(nbs[j]):
                    A[j, j] += cval[j, k]
                    if nn is not None:
                        A[j, nn] -= cval[j, k]
            xv = np.linalg.solve(A, bv)
        else:
            xv = bv * (1.0 + 1e-3 * rng.normal(size=N))
        x = [split(v) for v in xv]
        b = [split(v) for v in bv]
        for j in range(N):
            cf = [split(v) for v in cval[j]]
            r = pair_tab_residual(x, b, j, nbs[j], cf)
            xj = exact(x[j])
            ex = exact(b[j]) - xj
            scale = abs(xj)
            for k, nn in enumerate(nbs[j]):
                xn = exact(x[nn]) if nn is not None else Fraction(0)
                ex -= exact(cf[k]) * (xj - xn)
                scale += exact(cf[k]) * (abs(xj) + abs(xn))
            err = abs(Fraction(float(r)) - ex)
            bound = 4 * scale / 2 ** 48 + abs(ex) / 2 ** 23
            assert err <= bound, (trial, j, float(err), float(bound))
            worst = max(worst, float((err - abs(ex) / 2 ** 23) / scale))
    assert worst <= 4 / 2 ** 48
