"""Coefficients of the Kerr-step polynomials in csrc/ldbp_tile.cuh.

Minimax (equal-ripple absolute error) approximations of sin x by an odd and
of cos x - 1 by an even polynomial on [0, X], by the Remez exchange
algorithm in FP64: tier A (degree 5 / 6, X = 0.5) and tier B (degree 7 / 8,
X = 1.0).  Run it to print the coefficients and their maximum errors; it is
a maintenance tool and is not imported by the library.
"""
import numpy as np


def remez(f, powers, X, iters=100, grid=200001):
    """Coefficients a of sum_k a_k x**powers[k] minimising max |f - p| on [0, X]."""
    m = len(powers)
    ref = X * (1 - np.cos(np.pi * np.arange(m + 1) / m)) / 2
    ref[0] = X * 1e-3
    xs = np.linspace(X * 1e-4, X, grid)
    for _ in range(iters):
        A = np.array([[x ** q for q in powers] + [(-1.0) ** i] for i, x in enumerate(ref)])
        a = np.linalg.solve(A, f(ref))[:m]
        err = f(xs) - sum(ak * xs ** q for ak, q in zip(a, powers))
        cuts = np.concatenate([[0], np.where(np.diff(np.sign(err)) != 0)[0] + 1, [len(xs)]])
        ext = np.array([c0 + np.argmax(np.abs(err[c0:c1])) for c0, c1 in zip(cuts[:-1], cuts[1:])])
        if len(ext) > m:
            best = max(range(len(ext) - m), key=lambda s: np.min(np.abs(err[ext[s:s + m + 1]])))
            ref = xs[ext[best:best + m + 1]]
    return a, float(np.max(np.abs(err)))


def main():
    for tier, X, sp, cp in (("A", 0.5, [1, 3, 5], [2, 4, 6]), ("B", 1.0, [1, 3, 5, 7], [2, 4, 6, 8])):
        a, ea = remez(np.sin, sp, X)
        b, eb = remez(lambda x: np.cos(x) - 1.0, cp, X)
        print(f"tier {tier} |x| <= {X}: sin {[float(v) for v in a]} (max error {ea:.3g}); "
              f"cos - 1 {[float(v) for v in b]} (max error {eb:.3g})")


if __name__ == "__main__":
    main()
