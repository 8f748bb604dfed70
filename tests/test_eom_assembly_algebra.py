"""The regrouping of the equation-of-motion assembly (CPU).

For one receiver mu, the beta != mu terms of dGamma^mu_kl are linear in each pair's S^{-1},
Im Delta, Qr and Qi.  The CUDA assembly sums them in two passes: elementwise sums
D = sum_beta (w2 Qr + w3 Qi + w4 S^{-1} + w5 Im) and T = sum_beta (w0 S^{-1} + w1 Im), then the
sparse commutator terms against A applied once to T, A_kl sum_beta w2, and the pairs' F_imp
terms on the impurity modes' rows and columns.  This test evaluates, on random data, the
per-element form term by term (every pair's [Delta, F], Q + F and Delta, as the single-pass
assembly wrote them) and the two-pass form, and requires them to agree to rounding."""
import numpy as np


def _case(rng, n=12, M=5, imp=(2, 7, 9)):
    A = rng.standard_normal((n, n)) * (rng.random((n, n)) < 0.25)
    A = A - A.T
    pairs = [(a, b) for a in range(M) for b in range(a + 1, M)]
    P = len(pairs)
    ni = len(imp)
    return dict(
        n=n, M=M, imp=list(imp), A=A, pairs=pairs,
        si=rng.standard_normal((P, n, n)), im=rng.standard_normal((P, n, n)),
        qr=rng.standard_normal((P, n, n)), qi=rng.standard_normal((P, n, n)),
        fimp=rng.standard_normal((P, ni, ni, 2)), coef=rng.standard_normal((M, M, 6)))


def _single_pass(c, mu):
    """Every beta != mu term per element, as the one-pass kernel formed it."""
    n, imp, A = c["n"], c["imp"], c["A"]
    slot = {m: i for i, m in enumerate(imp)}
    out = np.zeros((n, n))
    for p, (a, b) in enumerate(c["pairs"]):
        if mu not in (a, b):
            continue
        be = b if mu == a else a
        sgn = -1.0 if mu == a else 1.0
        s, im, fp, co = c["si"][p], c["im"][p], c["fimp"][p], c["coef"][mu, be]
        for k in range(n):
            for l in range(n):
                sk, sl = slot.get(k, -1), slot.get(l, -1)
                dre = lambda r, q: -2.0 * s[r, q]
                dim = lambda r, q: sgn * im[r, q]
                Dx, Dy = dre(k, l), dim(k, l)
                Fx, Fy = A[k, l], 0.0
                if sk >= 0 and sl >= 0:
                    Fx += fp[sk, sl, 0]
                    Fy += sgn * fp[sk, sl, 1]
                ss = -sum(s[k, q] * A[l, q] for q in range(n)) - sum(A[k, q] * s[q, l] for q in range(n))
                si_ = -sum(im[k, q] * A[l, q] for q in range(n)) - sum(A[k, q] * im[q, l] for q in range(n))
                dfx, dfy, fdx, fdy = -2.0 * ss, sgn * si_, 0.0, 0.0
                if sl >= 0:
                    for m, mm in enumerate(imp):
                        ax, ay = dre(k, mm), dim(k, mm)
                        bx, by = fp[m, sl, 0], sgn * fp[m, sl, 1]
                        dfx += ax * bx - ay * by
                        dfy += ax * by + ay * bx
                if sk >= 0:
                    for m, mm in enumerate(imp):
                        ax, ay = fp[sk, m, 0], sgn * fp[sk, m, 1]
                        bx, by = dre(mm, l), dim(mm, l)
                        fdx += ax * bx - ay * by
                        fdy += ax * by + ay * bx
                Cx, Cy = dfx - fdx, dfy - fdy
                QFx, QFy = c["qr"][p][k, l] + Fx, sgn * c["qi"][p][k, l] + Fy
                out[k, l] += 2.0 * (co[0] * Cx - co[1] * Cy + co[2] * QFx - co[3] * QFy + co[4] * Dx - co[5] * Dy)
    return out


def _two_pass(c, mu, drop_w1=False):
    """D and T summed elementwise, then the sparse part, A_kl sum w2 and the impurity terms
    (drop_w1: a planted mistake, T without its Im Delta part)."""
    n, imp, A = c["n"], c["imp"], c["A"]
    slot = {m: i for i, m in enumerate(imp)}
    D, T, w2sum = np.zeros((n, n)), np.zeros((n, n)), 0.0
    for p, (a, b) in enumerate(c["pairs"]):
        if mu not in (a, b):
            continue
        be = b if mu == a else a
        sgn = -1.0 if mu == a else 1.0
        co = c["coef"][mu, be]
        w = [-4 * co[0], -2 * sgn * co[1], 2 * co[2], -2 * sgn * co[3], -4 * co[4], -2 * sgn * co[5]]
        T += w[0] * c["si"][p] + (0.0 if drop_w1 else w[1]) * c["im"][p]
        D += w[2] * c["qr"][p] + w[3] * c["qi"][p] + w[4] * c["si"][p] + w[5] * c["im"][p]
        w2sum += w[2]
    out = D + A * w2sum - T @ A.T - A @ T
    for p, (a, b) in enumerate(c["pairs"]):       # impurity rows and columns
        if mu not in (a, b):
            continue
        be = b if mu == a else a
        sgn = -1.0 if mu == a else 1.0
        s, im, fp, co = c["si"][p], c["im"][p], c["fimp"][p], c["coef"][mu, be]
        for k in range(n):
            for l in range(n):
                sk, sl = slot.get(k, -1), slot.get(l, -1)
                if sk < 0 and sl < 0:
                    continue
                dfx = dfy = fdx = fdy = Fx = Fy = 0.0
                if sl >= 0:
                    for m, mm in enumerate(imp):
                        ax, ay = -2.0 * s[k, mm], sgn * im[k, mm]
                        bx, by = fp[m, sl, 0], sgn * fp[m, sl, 1]
                        dfx += ax * bx - ay * by
                        dfy += ax * by + ay * bx
                if sk >= 0:
                    for m, mm in enumerate(imp):
                        ax, ay = fp[sk, m, 0], sgn * fp[sk, m, 1]
                        bx, by = -2.0 * s[mm, l], sgn * im[mm, l]
                        fdx += ax * bx - ay * by
                        fdy += ax * by + ay * bx
                if sk >= 0 and sl >= 0:
                    Fx, Fy = fp[sk, sl, 0], sgn * fp[sk, sl, 1]
                out[k, l] += 2.0 * (co[0] * (dfx - fdx) - co[1] * (dfy - fdy) + co[2] * Fx - co[3] * Fy)
    return out


def test_two_pass_assembly_equals_the_per_element_form():
    rng = np.random.default_rng(17)
    c = _case(rng)
    for mu in range(c["M"]):
        ref = _single_pass(c, mu)
        got = _two_pass(c, mu)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), mu


def test_a_dropped_weight_is_caught():
    """The comparison is sharp: T without its Im Delta part disagrees."""
    rng = np.random.default_rng(18)
    c = _case(rng)
    ref = _single_pass(c, 1)
    got = _two_pass(c, 1, drop_w1=True)
    assert np.abs(got - ref).max() > 1e-6 * np.abs(ref).max()
