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


def test_noalloc_allocates_no_device_memory(env):
    """After a first call on the device (which loads its kernels), a call leaves the
    device's free memory unchanged: the only scratch is the file-scope array."""
    fc, torch, w, ctx, gid, t = env
    pts = torch.tensor([11, 2222, 8888], dtype=torch.int64, device="cuda")
    out = torch.empty((3, 64, w.n_fit), dtype=torch.float32, device="cuda")
    fc.fc_fake_data_noalloc(t["S"], t["F"], pts, 5, 64, out, collapse=t["coll"], n_fit=w.n_fit)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    fc.fc_fake_data_noalloc(t["S"], t["F"], pts, 6, 64, out, collapse=t["coll"], n_fit=w.n_fit)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_more_points_than_one_grid_dimension(env):
    """P above 65535 (possible within the scratch limit when N_full is small) is split
    over several launches; the counts equal fc_fake_data's."""
    fc, torch, w, ctx, gid, t = env
    rng = np.random.default_rng(3)
    G, P, U = 500, 70000, 2
    S1 = rng.uniform(50.0, 500.0, (G, 1))
    F1 = np.array([[0.01]])
    pts = rng.integers(0, G, P).astype(np.int64)
    g1 = fc.fc_load_grid(ctx, S1)
    fc.fc_set_frac_cov(ctx, g1, F1)
    ref = fc.fc_fake_data(ctx, g1, pts, 9, U, 1)
    out = torch.full((P, U, 1), -1.0, dtype=torch.float32, device="cuda")
    fc.fc_fake_data_noalloc(torch.from_numpy(S1).cuda(), torch.from_numpy(F1).cuda(), torch.from_numpy(pts).cuda(), 9,
                            U, out)
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    fc.fc_unload_grid(ctx, g1)


@pytest.mark.parametrize("bad", ["negative", "too_large", "empty_bin"])
def test_noalloc_rejects_bad_collapse_map(env, bad):
    fc, torch, w, ctx, gid, t = env
    coll = w.collapse.copy()
    if bad == "negative":
        coll[7] = -1
    elif bad == "too_large":
        coll[7] = w.n_fit
    else:
        coll[1] = coll[0] = 0  # full bins 0 and 1 both to fit bin 0 ...
        coll[2] = coll[3] = 0  # ... and fit bin 1 gets nothing
    ps = torch.tensor([1, 2], dtype=torch.int64, device="cuda")
    out = torch.empty((2, 2, w.n_fit), dtype=torch.float32, device="cuda")
    with pytest.raises(fc.FCError) as e:
        fc.fc_fake_data_noalloc(t["S"], t["F"], ps, 1, 2, out, collapse=torch.from_numpy(coll).cuda(), n_fit=w.n_fit)
    assert e.value.status == fc.FC_ERR_ARG
