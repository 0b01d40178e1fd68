"""The allocation-free table build, through the C ABI, against the context path.

acc_motif_build_table_static is for callers that cannot allocate device
memory where they need the table (a fixed memory budget, a framework that owns
the allocator, a stream under graph capture).  It writes into buffers the
caller owns and works in a fixed array inside the library.  Its output must
equal the CPU oracle's table and class codes and those of the ordinary entry
points, on two calls in a row (the shared array keeps the previous call's
contents).

This file is named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def acc():
    import torch  # noqa: F401
    from paper_1203_3415_gb300 import build
    build.build()
    import paper_1203_3415_gb300 as p
    return p


def test_static_table_matches_context_table(acc):
    import oracle
    import torch
    counter = acc.Counter(0)
    stream = torch.cuda.current_stream()
    for k in (5, 3, 4):
        want_table = counter.table(k)
        want_codes = np.array([counter.class_code(k, c) for c in range(acc.NUM_CLASSES[k])], dtype=np.int64)
        # the CPU oracle's own table and class codes, written independently
        o_table, o_codes = oracle.table(k)
        assert np.array_equal(want_table, np.asarray(o_table, np.int16)), k
        assert np.array_equal(want_codes, np.asarray(o_codes, np.int64)), k
        for call in range(2):
            table = torch.full((1 << (k * (k - 1)),), 77, dtype=torch.int16, device="cuda")
            # a sentinel no canonical code can take: every class slot must be written
            codes = torch.full((acc.NUM_CLASSES[k],), -1, dtype=torch.int32, device="cuda")
            rc = acc.acc_motif_build_table_static(k, stream.cuda_stream, table.data_ptr(), codes.data_ptr())
            assert rc == acc.ACC_OK, acc.acc_strerror(rc)
            torch.cuda.synchronize()
            got = table.cpu().numpy()
            assert int(got.min()) >= -1 and int(got.max()) == acc.NUM_CLASSES[k] - 1, (k, call)
            assert np.array_equal(got, want_table), (k, call)
            assert np.array_equal(got, np.asarray(o_table, np.int16)), (k, call)
            got_codes = codes.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
            assert not np.any(got_codes == 0xFFFFFFFF), (k, call)
            assert np.array_equal(got_codes, want_codes), (k, call)
            assert np.array_equal(got_codes, np.asarray(o_codes, np.int64)), (k, call)
    counter.close()


def test_static_table_rejects_bad_arguments(acc):
    import torch
    table = torch.zeros(64, dtype=torch.int16, device="cuda")
    codes = torch.zeros(13, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert acc.acc_motif_build_table_static(6, s, table.data_ptr(), codes.data_ptr()) == acc.ACC_ERR_K
    assert acc.acc_motif_build_table_static(2, s, table.data_ptr(), codes.data_ptr()) == acc.ACC_ERR_K
    assert acc.acc_motif_build_table_static(3, s, 0, codes.data_ptr()) == acc.ACC_ERR_ARG
    assert acc.acc_motif_build_table_static(3, s, table.data_ptr(), 0) == acc.ACC_ERR_ARG
