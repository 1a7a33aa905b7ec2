"""GPU check of bie_rotate_noalloc, the rotation entry point for callers that cannot allocate device
memory (frameworks that own all device memory, loops that must not touch the allocator).  It must give the same rotated coefficients as bie_rotate, on consecutive calls that reuse
its fixed staging array, and reject requests too large for that array before touching the GPU.
This file is collected last so that a failure here cannot hide the result of any other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1707_02156_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12  # the FP64 tolerance of the other GPU parity tests


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_02156_gb300 import api, build
    build.build()
    return api.Context(0)


def _relerr(a, b):
    a, b = a.ravel(), b.ravel()
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_rotate_noalloc_matches_rotate_on_two_calls_in_a_row(ctx):
    rng = np.random.default_rng(2024)
    calls = [([5, 16, 32], 3, [(0.3, 1.1, -0.4), (2.0, 2.9, 0.0), (-1.2, 0.05, 1.7)]),
             ([24, 7], 2, [(1.4, 0.6, 0.2), (-2.5, 2.2, -1.0)])]
    for ps, ncomp, eul in calls:
        coefs = [inputs.random_bandlimited(rng, p, ncomp, decay_pow=0.5) for p in ps]
        c = torch.as_tensor(np.concatenate([x.ravel() for x in coefs])).cuda()
        ref = torch.zeros_like(c)
        got = torch.full_like(c, np.nan)
        ctx.rotate(ps, ncomp, c, eul, ref)
        ctx.rotate_noalloc(ps, ncomp, c, eul, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert _relerr(g, r) < FP64_TOL


def test_rotate_noalloc_rejects_degree_beyond_its_array(ctx):
    from paper_1707_02156_gb300 import api
    c = torch.zeros(3 * 66 * 66, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(c)
    with pytest.raises(api.BIEError) as e:
        ctx.rotate_noalloc([65], 3, c, [(0.1, 0.2, 0.3)], out)
    assert e.value.status == 1 and "BIE_NOALLOC_MAX_P" in str(e.value)
