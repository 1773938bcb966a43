"""tsne_kl_noalloc: the KL entry point for callers that cannot allocate device
memory (its scratch is a fixed array in the library's device image). It must
give the plan-based tsne_kl's value, call after call: the second call checks
that the shared scratch is reset between calls. Collected last on purpose."""
import numpy as np
import pytest
import torch

import paper_1712_09005_gb300 as pkg
from paper_1712_09005_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("s", [1, 2])
def test_kl_noalloc_matches_plan_kl_twice(s):
    N = 3001
    X = inputs.mixture(N=N, n_clusters=5, seed=77)
    P = inputs.affinities(X, 30.0, device="cpu")
    rng = np.random.default_rng(5 + s)
    Pd = pkg.DeviceCSR.from_host(*P.as_tuple())
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pkg.Plan(N, s) as plan:
        for call in range(2):
            Y = torch.as_tensor(rng.normal(0, 10, size=(N, s)).astype(np.float32), device="cuda")
            want = plan.kl(Pd, Y)  # also leaves this Y's Z in the plan
            Z = plan.info()["Z"]
            out.fill_(float("nan"))
            pkg.tsne_kl_noalloc(Pd, Y, s, Z, out)
            torch.cuda.synchronize()
            got = float(out.item())
            # same kernel arithmetic with a different number of reduction blocks:
            # equal up to FP64 summation order
            assert abs(got - want) <= 1e-12 * abs(want), (call, got, want)


def test_kl_noalloc_rejects_bad_sizes():
    Pd = pkg.DeviceCSR.from_host(np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32),
                                 np.array([0.5, 0.5], np.float32))
    Y = torch.zeros((2, 2), device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.TsneError):
        pkg.tsne_kl_noalloc(Pd, Y, 3, 1.0, out)
    with pytest.raises(pkg.TsneError):
        pkg.tsne_kl_noalloc(Pd, Y, 2, 0.0, out)


def test_kl_noalloc_rejects_mismatched_y():
    """Y must hold P's N points as contiguous float32 on the device: a Y with
    fewer rows than P (the kernel would read past its end), a float64 Y and a
    host Y are rejected before the call."""
    Pd = pkg.DeviceCSR.from_host(np.array([0, 1, 2, 2], np.int32), np.array([1, 0], np.int32),
                                 np.array([0.5, 0.5], np.float32))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        pkg.tsne_kl_noalloc(Pd, torch.zeros((2, 2), device="cuda"), 2, 1.0, out)
    with pytest.raises(TypeError):
        pkg.tsne_kl_noalloc(Pd, torch.zeros((3, 2), dtype=torch.float64, device="cuda"), 2, 1.0, out)
    with pytest.raises(TypeError):
        pkg.tsne_kl_noalloc(Pd, torch.zeros((3, 2)), 2, 1.0, out)
