"""soft_step_noalloc -- the step entry point for callers that cannot allocate
device memory while stepping -- must give the same state as soft_step, call
after call, and must refuse requests larger than its fixed scratch.

Collected last on purpose (file name): if it fails, a run that stops at the
first failure has already run every other test.  It passes both alone in a
fresh process and after the other tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_1505_06707_gb300 as S  # noqa: E402

TOL = {S.SOFT_C128: 1e-11, S.SOFT_C64: 1e-5}


@pytest.mark.parametrize("prec", [S.SOFT_C128, S.SOFT_C64])
def test_noalloc_matches_soft_step_twice(prec):
    assert torch.cuda.is_available()
    n, a, b, R0 = 2048, -16.0, 16.0, 12.0
    x = a + (b - a) / n * (np.arange(n) + 0.5)
    psi0 = np.exp(-(x - 1.0) ** 2 / 2.0 + 0.4j * x)
    field = (0.05, 0.057, 4.0)
    ct = torch.complex64 if prec == S.SOFT_C64 else torch.complex128
    plan = S.soft_create(n, (a, b), R0, 0.5, 0.02, prec=prec, contour=S.CONTOUR_SECS)
    try:
        ref = torch.tensor(psi0, dtype=ct, device="cuda")
        got = torch.tensor(psi0, dtype=ct, device="cuda")
        t_ref = t_got = 10.0
        for _ in range(2):                       # two calls in a row
            t_ref = S.soft_step(plan, ref, 150, t_ref, field=field)
            t_got = S.soft_step_noalloc(plan, got, 150, t_got, field=field)
            torch.cuda.synchronize()
            r = ref.cpu().numpy().astype(np.complex128)
            g = got.cpu().numpy().astype(np.complex128)
            assert abs(t_ref - t_got) < 1e-12
            assert np.linalg.norm(g - r) / np.linalg.norm(r) < TOL[prec]
        with pytest.raises(S.SoftError) as e:
            S.soft_step_noalloc(plan, got, 16385, t_got, field=field)
        assert e.value.status == -11
    finally:
        S.soft_destroy(plan)
