"""Shared helpers of the GPU tests: build problems through the C ABI binding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

needs_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")


def lib():
    from paper_1703_10016_gb300 import igs
    return igs


class Prob:
    """One geometry + problem on a context, destroyed on close."""

    def __init__(self, ctx, curve, n_elems, degree, n_ref, precision):
        g = lib()
        self.g = g
        self.geom = g.igs_create_geometry(ctx, curve.degree, curve.knots, curve.ctrl, curve.weights, curve.closed)
        self.prob = g.igs_create_problem(self.geom, degree, n_elems, n_ref, precision)
        self.info = g.igs_problem_info(self.prob)

    def assemble(self, dtype=np.float64):
        n = self.info.n
        A = np.empty((n, n), dtype=dtype)
        self.g.igs_assemble(self.prob, A)
        return A

    def dense_W(self):
        eta, wb, first, _ = self.g.igs_get_rules(self.prob)
        n = self.info.n
        W = np.zeros((self.info.n_quad, n))
        for m in range(self.info.n_quad):
            for r in range(wb.shape[1]):
                if wb[m, r] != 0.0:
                    W[m, (first[m] + r) % n] += wb[m, r]
        return eta, W

    def close(self):
        self.g.igs_destroy_problem(self.prob)
        self.g.igs_destroy_geometry(self.geom)


def relF(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
