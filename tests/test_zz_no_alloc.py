"""The allocation-free write-back entry point, icd2s_apply_flips_static.

It serves callers that cannot call cudaMalloc (their device memory belongs
to a host framework or another allocator, or they must not allocate while
running): it works on buffers the caller owns and keeps its own scratch in a
static device array.  Here it is called through the C ABI on caller-owned
torch buffers and must give exactly what the handle-based
icd2s_apply_flips_update_gains gives on the same inputs, and the oracle's
gains and energies of the new solutions, on two calls in a row (the static
scratch keeps the previous call's contents, so the second call checks that
it starts clean).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2502_13947_gb300 import build as B
from paper_2502_13947_gb300 import icd2s as I
from paper_2502_13947_gb300.instances import make_qubo, random_solutions

from .gpu_util import dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,ld,R", [(777, 784, 5), (777, 780, 5), (1000, 1000, 3), (2499, 2500, 8),
                                    (2500, 2560, 8)])
def test_static_write_back_equals_the_handle_based_one(orc, n, ld, R):
    """Row strides that are multiples of 16 (16-byte path) and of 4 only
    (4-byte path: 780 and 2500 also end inside a 4-column group and, at 2500,
    span three column tiles).  The second call runs on an explicit stream.
    The caller's padding columns of Q, x and g hold non-zero values: Q's are
    never used for the result, x's and g's are left as they were."""
    torch = torch_cuda()
    B.build()
    Q = make_qubo(n, 0.3, n)
    X0 = random_solutions(n, R, 1)
    rng = np.random.default_rng(n + ld)
    M1 = (rng.random((R, n)) < 0.05).astype(np.uint8)
    M2 = (rng.random((R, n)) < 0.2).astype(np.uint8)
    M1[0] = 0                       # a replica with nothing to flip
    M2[-1] = 1                      # a replica where everything flips

    # the existing entry point, on library-owned state
    q = I.icd2s_qubo_create(Q)
    st = I.icd2s_state_create(q, R, 3)
    I.icd2s_state_load(st, X0)
    _, g0, E0 = I.icd2s_get_state(st, R, n)
    M1d, M2d = dev(M1), dev(M2)
    I.icd2s_apply_flips_update_gains(st, M1d.data_ptr())
    want1 = I.icd2s_get_state(st, R, n)
    I.icd2s_apply_flips_update_gains(st, M2d.data_ptr())
    want2 = I.icd2s_get_state(st, R, n)
    I.icd2s_state_destroy(st)
    I.icd2s_qubo_destroy(q)

    # the static entry point, on caller-owned buffers with row stride ld
    Qp = rng.integers(-100, 101, (n, ld)).astype(np.int8)
    Qp[:, :n] = Q
    Xp = np.full((R, ld), 7, np.uint8)
    Xp[:, :n] = X0
    Gp = np.full((R, ld), -12345, np.int32)
    Gp[:, :n] = g0
    Qd, Xd, Gd, Ed = dev(Qp), dev(Xp), dev(Gp), dev(E0.copy())
    side = torch.cuda.Stream()
    for call, (M_d, (wx, wg, wE)) in enumerate(((M1d, want1), (M2d, want2))):
        if call == 0:
            I.icd2s_apply_flips_static(Qd.data_ptr(), n, ld, R, M_d.data_ptr(), Xd.data_ptr(), Gd.data_ptr(),
                                       Ed.data_ptr())
            torch.cuda.synchronize()
        else:
            side.wait_stream(torch.cuda.current_stream())
            I.icd2s_apply_flips_static(Qd.data_ptr(), n, ld, R, M_d.data_ptr(), Xd.data_ptr(), Gd.data_ptr(),
                                       Ed.data_ptr(), stream=side.cuda_stream)
            side.synchronize()
        x, g, E = Xd.cpu().numpy(), Gd.cpu().numpy(), Ed.cpu().numpy()
        assert np.array_equal(x[:, :n], wx)
        assert np.array_equal(g[:, :n], wg)
        assert np.array_equal(E, wE)
        assert (x[:, n:] == 7).all() and (g[:, n:] == -12345).all()
        # and against the oracle's definition-level gains and energies (Eq. 1)
        assert np.array_equal(E, orc.energy_batch(Q, np.ascontiguousarray(x[:, :n])))
        for p in (0, R - 1):
            assert np.array_equal(g[p, :n], orc.gains(Q, np.ascontiguousarray(x[p, :n])))


def test_static_write_back_rejects_sizes_beyond_its_scratch():
    torch = torch_cuda()
    B.build()
    n, ld, R = 4096, 4096, 300          # 300 * 4096 > 2^20 flip-list entries
    Qd = torch.zeros((n, ld), dtype=torch.int8, device="cuda")
    Md = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    Xd = torch.zeros((R, ld), dtype=torch.uint8, device="cuda")
    Gd = torch.zeros((R, ld), dtype=torch.int32, device="cuda")
    Ed = torch.zeros(R, dtype=torch.int64, device="cuda")
    with pytest.raises(I.ICD2SError) as e:
        I.icd2s_apply_flips_static(Qd.data_ptr(), n, ld, R, Md.data_ptr(), Xd.data_ptr(), Gd.data_ptr(),
                                   Ed.data_ptr())
    assert e.value.code == I.ERR_RANGE and "static scratch" in str(e.value)
