"""The allocation-free fake-data entry point (fc_fake_data_noalloc).

It exists for callers that cannot allocate device memory where they need fake
data (code inside another framework's allocator callback, request paths that
must not allocate after start-up).  Its output must equal fc_fake_data's -- bit for bit,
the fake-data tolerance used everywhere else -- on consecutive calls that
share its static scratch.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import paper_2002_07858_gb300 as fc

    fc.load()
    w = workloads.cfg2()
    ctx = fc.fc_create(0)
    gid = fc.fc_load_grid(ctx, w.S, w.collapse, w.n_fit)
    fc.fc_set_frac_cov(ctx, gid, w.F)
    dev = torch.device("cuda", 0)
    t = dict(S=torch.from_numpy(w.S).to(dev), F=torch.from_numpy(w.F).to(dev),
             coll=torch.from_numpy(w.collapse).to(dev))
    yield fc, torch, w, ctx, gid, t
    fc.fc_destroy(ctx)


def test_noalloc_matches_fc_fake_data_on_consecutive_calls(env):
    fc, torch, w, ctx, gid, t = env
    U = 300
    stream = torch.cuda.current_stream().cuda_stream
    for pts, seed in ((np.array([0, 1234, 5555, 9999], np.int64), 7),
                      (np.array([42, 77, 4242], np.int64), 8)):
        ref = fc.fc_fake_data(ctx, gid, pts, seed, U, w.n_fit)
        out = torch.full((len(pts), U, w.n_fit), -1.0, dtype=torch.float32, device="cuda")
        ps = torch.from_numpy(pts).cuda()
        fc.fc_fake_data_noalloc(t["S"], t["F"], ps, seed, U, out, collapse=t["coll"], n_fit=w.n_fit,
                                cuda_stream=stream)
        np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    fc, torch, w, ctx, gid, t = env
    P = 400  # 400 * 90^2 * 12 bytes > 16 MiB
    ps = torch.zeros(P, dtype=torch.int64, device="cuda")
    out = torch.empty((P, 2, w.n_fit), dtype=torch.float32, device="cuda")
    with pytest.raises(fc.FCError) as e:
        fc.fc_fake_data_noalloc(t["S"], t["F"], ps, 1, 2, out, collapse=t["coll"], n_fit=w.n_fit)
    assert e.value.status == fc.FC_ERR_ARG and "16 MiB" in str(e.value)


def test_noalloc_rejects_bad_point_index(env):
    fc, torch, w, ctx, gid, t = env
    ps = torch.tensor([0, w.G], dtype=torch.int64, device="cuda")
    out = torch.empty((2, 2, w.n_fit), dtype=torch.float32, device="cuda")
    with pytest.raises(fc.FCError) as e:
        fc.fc_fake_data_noalloc(t["S"], t["F"], ps, 1, 2, out, collapse=t["coll"], n_fit=w.n_fit)
    assert e.value.status == fc.FC_ERR_ARG
