"""GPU parity: the CUDA path, called through the C ABI, against the FP64
oracle on the same seeded complex64 inputs (promoted to FP64 for the
oracle).  Tolerance: relative L2 error <= 2e-6 per transform, the bound the
plain FP32 path must meet at every size."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 2e-6


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0811_2535_gb300 import build, moafft
    build.build()
    import oracle
    oracle.build()
    return torch, moafft, oracle


def per_transform_rel(y, ref, batch):
    y = np.asarray(y, np.complex128).reshape(batch, -1)
    ref = np.asarray(ref, np.complex128).reshape(batch, -1)
    return np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)


def run(env, shape, batch, sign, x, inplace=False, adjoint=False):
    torch, moafft, _ = env
    plan = moafft.Plan(shape, batch, sign)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    if inplace:
        out = plan.exec_adjoint(xd, out=xd) if adjoint else plan.exec(xd, out=xd)
    else:
        out = plan.exec_adjoint(xd) if adjoint else plan.exec(xd)
    y = out.cpu().numpy()
    assert plan.status() == 0
    info = plan.info()
    plan.destroy()
    return y, info


def oracle_ref(env, x, shape, batch, sign):
    _, _, oracle = env
    x64 = np.asarray(x, np.complex128).reshape((batch,) + tuple(shape))
    if len(shape) == 1:
        return oracle.fft_radix2(x64, sign)
    return oracle.fft_nd(x64, len(shape), sign)


@pytest.mark.parametrize("t", range(1, 25))
@pytest.mark.parametrize("sign", [-1, 1])
def test_1d_every_size(env, t, sign):
    from paper_0811_2535_gb300 import inputs
    n = 1 << t
    x = inputs.uniform(n, 1000 + t)
    y, info = run(env, [n], 1, sign, x)
    err = per_transform_rel(y, oracle_ref(env, x, [n], 1, sign), 1).max()
    assert err <= TOL, (n, err)
    assert info["passes"] == (1 if t <= 12 else 2)


@pytest.mark.parametrize("n,batch", [(2, 3), (16, 5), (32, 7), (1024, 5), (4096, 3), (8192, 3), (1 << 16, 5),
                                     (1 << 20, 2)])
def test_1d_batched_ragged(env, n, batch):
    from paper_0811_2535_gb300 import inputs
    x = inputs.uniform((batch, n), 2000 + n + batch)
    y, _ = run(env, [n], batch, -1, x)
    err = per_transform_rel(y, oracle_ref(env, x, [n], batch, -1), batch)
    assert err.max() <= TOL, err


@pytest.mark.parametrize("t", [13, 14, 17, 20, 24])
def test_1d_every_split(env, t, monkeypatch):
    """Sec. 4.8: any breakpoint (here: any r x c split) gives the same result."""
    from paper_0811_2535_gb300 import inputs
    n = 1 << t
    x = inputs.uniform(n, 3000 + t)
    ref = oracle_ref(env, x, [n], 1, -1)
    for lr in range(max(1, t - 12), min(12, t - 1) + 1):
        monkeypatch.setenv("MOA_SPLIT_LOG2R", str(lr))
        y, info = run(env, [n], 1, -1, x)
        assert info["split_r"] == 1 << lr
        err = per_transform_rel(y, ref, 1).max()
        assert err <= TOL, (lr, err)


@pytest.mark.parametrize("shape,batch", [((1 << 10,), 1), ((1 << 16,), 2), ((64, 32), 3), ((4096, 4096), 1),
                                         ((16, 8, 4), 2), ((256, 256, 256), 1)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_in_place(env, shape, batch, sign):
    from paper_0811_2535_gb300 import inputs
    x = inputs.uniform((batch,) + shape, 4000 + len(shape))
    y, _ = run(env, list(shape), batch, sign, x, inplace=True)
    err = per_transform_rel(y, oracle_ref(env, x, list(shape), batch, sign), batch)
    assert err.max() <= TOL, err


@pytest.mark.parametrize("shape,batch", [((2, 2), 1), ((2, 4096), 1), ((4096, 2), 1), ((8, 16), 5), ((512, 128), 2),
                                         ((4, 8, 16), 3), ((2, 2, 2), 2), ((64, 2, 128), 1), ((32, 64, 16), 2)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_nd_shapes(env, shape, batch, sign):
    from paper_0811_2535_gb300 import inputs
    x = inputs.uniform((batch,) + shape, 5000 + sum(shape))
    y, _ = run(env, list(shape), batch, sign, x)
    err = per_transform_rel(y, oracle_ref(env, x, list(shape), batch, sign), batch)
    assert err.max() <= TOL, err


def test_config_small_forward_and_round_trip(env):
    """n = 2^10, batch 1, seed 0: forward and the inverse round trip."""
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << 10
    x = inputs.uniform(n, inputs.SEED_SMALL)
    plan = moafft.Plan([n], 1, -1)
    X = plan.exec(torch.from_numpy(x).cuda())
    back = plan.exec_adjoint(X).cpu().numpy() / n
    ref = oracle.fft_radix2(x.astype(np.complex128), -1)
    assert per_transform_rel(X.cpu().numpy(), ref, 1).max() <= TOL
    assert per_transform_rel(back, x, 1).max() <= TOL


@pytest.mark.parametrize("shape", [(1 << 24,), (4096, 4096), (256, 256, 256)])
def test_config_large_full_size(env, shape):
    """The full-size workloads (seed 1), every output element vs the oracle,
    in the launch configuration the benchmark times."""
    from paper_0811_2535_gb300 import inputs
    x = inputs.uniform(shape, inputs.SEED_LARGE)
    y, info = run(env, list(shape), 1, -1, x)
    ref = oracle_ref(env, x, list(shape), 1, -1)
    err = per_transform_rel(y, ref, 1).max()
    assert err <= TOL, err
    # elementwise: no single output far off relative to the transform's scale
    scale = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(y.reshape(-1) - ref.reshape(-1))) <= 50 * TOL * scale
    if len(shape) == 1:
        assert (info["split_r"], info["split_c"]) == (4096, 4096)


def test_adjoint_identity_and_round_trip(env):
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    for n in (1 << 9, 1 << 18):
        x = inputs.uniform(n, 11)
        z = inputs.uniform(n, 12)
        plan = moafft.Plan([n], 1, -1)
        Fx = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.complex128)
        FHz = plan.exec_adjoint(torch.from_numpy(z).cuda()).cpu().numpy().astype(np.complex128)
        lhs = np.vdot(z.astype(np.complex128), Fx)
        rhs = np.vdot(FHz, x.astype(np.complex128))
        assert abs(lhs - rhs) / abs(lhs) < 1e-5
        back = plan.exec_adjoint(plan.exec(torch.from_numpy(x).cuda())).cpu().numpy() / n
        assert per_transform_rel(back, x, 1).max() <= TOL


def test_exec_host_end_to_end(env):
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << 16
    x = inputs.uniform(n, 13)
    plan = moafft.Plan([n], 1, -1)
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    dbuf = torch.empty(n, dtype=torch.complex64, device="cuda")
    plan.exec_host(hin, hout, dbuf)
    torch.cuda.current_stream().synchronize()
    ref = oracle.fft_radix2(x.astype(np.complex128), -1)
    assert per_transform_rel(hout.numpy(), ref, 1).max() <= TOL


def test_exec_on_side_stream(env):
    torch, moafft, oracle = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << 14
    x = inputs.uniform((4, n), 14)
    plan = moafft.Plan([n], 4, -1)
    s = torch.cuda.Stream()
    xd = torch.from_numpy(x).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        y = plan.exec(xd, stream=s)
    s.synchronize()
    ref = oracle.fft_radix2(x.astype(np.complex128), -1)
    assert per_transform_rel(y.cpu().numpy(), ref, 4).max() <= TOL


@pytest.mark.parametrize("shape,batch", [((1 << 20,), 1), ((1 << 22,), 1), ((1 << 24,), 1), ((1 << 21,), 3),
                                         ((4096, 4096), 1), ((2048, 1024), 2), ((1024, 8), 3)])
def test_pipelined_and_generic_kernels_agree(env, shape, batch, monkeypatch):
    """The persistent TMA-pipelined strided kernels and the generic kernels
    compute the same transform (both checked against the oracle)."""
    from paper_0811_2535_gb300 import inputs
    x = inputs.uniform((batch,) + shape, 6000 + len(shape))
    ref = oracle_ref(env, x, list(shape), batch, -1)
    ys = []
    for pipe in ("2", "1", "0"):
        monkeypatch.setenv("MOA_PIPE", pipe)
        for sign in (-1,):
            y, _ = run(env, list(shape), batch, sign, x)
            assert per_transform_rel(y, ref, batch).max() <= TOL, pipe
            ys.append(y)
    assert per_transform_rel(ys[0], ys[2], batch).max() <= TOL
    assert per_transform_rel(ys[1], ys[2], batch).max() <= TOL


@pytest.mark.parametrize("L,lr,batch", [(24, 12, 1), (22, 11, 2), (20, 10, 3), (23, 12, 1), (23, 11, 2), (21, 10, 1)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_blocked_workspace_lifted(env, L, lr, batch, sign, monkeypatch):
    """Lifted 1-D with the intermediate in 4 x 4 blocks: pass 1 is the
    column kernel with block stores, pass 2 the column kernel reading the
    blocks through a 3-D tensor map; every r x c split with r, c >= 1024."""
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    monkeypatch.setenv("MOA_PIPE", "2")
    monkeypatch.setenv("MOA_SPLIT_LOG2R", str(lr))
    n = 1 << L
    x = inputs.uniform((batch, n), 6100 + L + lr)
    plan = moafft.Plan([n], batch, sign)
    names = [plan.pass_info(i)["kernel"] for i in range(plan.info()["passes"])]
    def pipe_col(logn, tw4, blk):   # two columns per thread at N = 4096
        return "pipe_col2_kernel<%d,%d>" % (tw4, blk) if logn == 12 else "pipe_col_kernel<%d,%d,%d>" % (logn, tw4, blk)
    assert names == [pipe_col(lr, 1, 1), pipe_col(L - lr, 0, 2)], names
    y = plan.exec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert plan.status() == 0
    plan.destroy()
    ref = oracle_ref(env, x, [n], batch, sign)
    assert per_transform_rel(y, ref, batch).max() <= TOL


@pytest.mark.parametrize("L,batch", [(24, 1), (23, 2), (22, 1), (21, 3)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_three_level_lift(env, L, batch, sign, monkeypatch):
    """n = 256 x cA x cB: the r = 256 column pass, then the second and third
    pass fused in one work-queue launch (middle tiles in place, last tiles
    waiting on per-unit counters), against the oracle."""
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    monkeypatch.setenv("MOA_LIFT3", "1")
    n = 1 << L
    x = inputs.uniform((batch, n), 6200 + L)
    plan = moafft.Plan([n], batch, sign)
    la, lb = (L - 7) // 2, (L - 8) // 2
    names = [plan.pass_info(i)["kernel"] for i in range(plan.info()["passes"])]
    assert names == ["col_pass_kernel<8,1>", "lift3_kernel<%d,%d>" % (la, lb)], names
    xd = torch.from_numpy(x).cuda()
    y = plan.exec(xd).cpu().numpy()
    y2 = plan.exec(xd).cpu().numpy()          # the queue and counters are reset per exec
    assert plan.status() == 0
    plan.destroy()
    ref = oracle_ref(env, x, [n], batch, sign)
    assert per_transform_rel(y, ref, batch).max() <= TOL
    assert np.array_equal(y, y2)


def test_pdl_chain_across_plans(env, monkeypatch):
    """Every pass is a programmatic dependent launch of the kernel before it
    in the stream and waits for it on the device.  A chain of execs of
    different plans on one stream, each reading the buffer the previous one
    wrote and writing the buffer it read, gives the same bits as the same
    chain in plain stream order with a synchronize after every exec."""
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    n = 1 << 24
    x = torch.from_numpy(inputs.uniform((n,), 6400)).cuda()
    monkeypatch.setenv("MOA_AUTOTUNE", "0")
    specs = [([n], 1, -1, moafft.MOA_C64, {}), ([4096, 4096], 1, 1, moafft.MOA_C64, {}),
             ([256, 256, 256], 1, -1, moafft.MOA_C64, {}), ([1 << 20], 16, 1, moafft.MOA_C64, {}),
             ([4096], 4096, -1, moafft.MOA_C64_TC_FP16, {}), ([4096], 4096, 1, moafft.MOA_C64, {}),
             ([n], 1, -1, moafft.MOA_C64, {"MOA_LIFT3": "1"}), ([1 << 12, 1 << 12], 1, 1, moafft.MOA_C64, {})]
    plans = []
    for shape, batch, sign, dtype, envs in specs:
        for k, v in envs.items():
            monkeypatch.setenv(k, v)
        plans.append(moafft.Plan(shape, batch, sign, dtype))
        for k in envs:
            monkeypatch.delenv(k)

    def chain(pdl):
        monkeypatch.setenv("MOA_PDL", "1" if pdl else "0")
        a, b = x.clone(), torch.empty_like(x)
        for p in plans:
            p.exec(a, out=b)
            if not pdl:
                torch.cuda.synchronize()
            a, b = b, a
        torch.cuda.synchronize()
        return a.cpu().numpy()

    ref = chain(False)
    got = chain(True)
    again = chain(True)
    for p in plans:
        assert p.status() == 0
        p.destroy()
    assert np.isfinite(ref).all()
    assert np.array_equal(got, ref)
    assert np.array_equal(again, ref)


@pytest.mark.parametrize("shape,batch", [((1 << 24,), 1), ((4096, 4096), 1), ((256, 256, 256), 1), ((4096, 8), 2)])
def test_output_only_eight_byte_aligned(env, shape, batch):
    """A 16-byte aligned input with an output one complex64 past a 16-byte
    boundary.  1-D 2^24 and 3-D 256^3: the last pass reads the aligned
    workspace and writes the output through the four-column N = 4096 kernel
    (8-byte plain stores), whose arithmetic is that of the two-column one:
    the results equal those of the aligned output bit for bit.  2-D: the
    column pass reads the misaligned output in place, so the generic kernel
    runs.  Every case matches the oracle."""
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    n = int(np.prod(shape)) * batch
    x = inputs.uniform((batch,) + shape, 6700 + n % 991)
    xin = torch.from_numpy(x.reshape(-1)).cuda()
    assert xin.data_ptr() % 16 == 0
    bout = torch.empty(n + 1, dtype=torch.complex64, device="cuda")
    yout = bout[1:]
    assert yout.data_ptr() % 16 == 8
    plan = moafft.Plan(list(shape), batch, -1)
    plan.exec(xin, out=yout)
    aligned = plan.exec(xin).cpu().numpy()
    assert plan.status() == 0
    plan.destroy()
    y = yout.cpu().numpy()
    if len(shape) != 2:
        assert np.array_equal(y, aligned)
    assert per_transform_rel(y, oracle_ref(env, x, list(shape), batch, -1), batch).max() <= TOL


@pytest.mark.parametrize("shape,batch", [((1 << 24,), 1), ((1 << 22,), 2), ((1 << 20,), 3), ((1 << 13,), 5),
                                         ((4096, 4096), 1), ((256, 256, 256), 1), ((64, 32), 3)])
def test_eight_byte_aligned_buffers(env, shape, batch):
    """The ABI asks only for 8-byte aligned buffers.  With input and output one
    complex64 past a 16-byte boundary, the TMA kernels that need 16-byte
    alignment give way to the generic ones (and a blocked 1-D plan runs both
    passes in the natural layout), with the same results."""
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    n = int(np.prod(shape)) * batch
    x = inputs.uniform((batch,) + shape, 6600 + n % 997)
    bin_ = torch.empty(n + 1, dtype=torch.complex64, device="cuda")
    bout = torch.empty(n + 1, dtype=torch.complex64, device="cuda")
    xin, yout = bin_[1:], bout[1:]
    assert xin.data_ptr() % 16 == 8 and yout.data_ptr() % 16 == 8
    xin.copy_(torch.from_numpy(x.reshape(-1)))
    plan = moafft.Plan(list(shape), batch, -1)
    plan.exec(xin, out=yout)
    y = yout.cpu().numpy()
    yin = bin_[1:]       # in place, also 8-byte aligned
    plan.exec(yin, out=yin)
    assert plan.status() == 0
    plan.destroy()
    ref = oracle_ref(env, x, list(shape), batch, -1)
    assert per_transform_rel(y, ref, batch).max() <= TOL
    assert per_transform_rel(yin.cpu().numpy(), ref, batch).max() <= TOL


@pytest.mark.parametrize("shape,batch", [((1 << 24,), 1), ((4096, 4096), 1), ((256, 256, 256), 1), ((1 << 20,), 3)])
def test_cuda_graph_of_dependent_launches(env, shape, batch):
    """Execs whose passes are programmatic dependent launches, captured in a
    CUDA graph (two execs back to back, so the second one's first pass
    depends on the first one's last) and replayed twice, give the same bits
    as the same execs run directly."""
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    x = torch.from_numpy(inputs.uniform((batch,) + shape, 6700 + len(shape))).cuda()
    plan = moafft.Plan(list(shape), batch, -1)
    inv = moafft.Plan(list(shape), batch, 1)
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    plan.exec(x, y1)
    inv.exec(y1, y2)
    torch.cuda.synchronize()
    ref1, ref2 = y1.clone(), y2.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.exec(x, y1)
        inv.exec(y1, y2)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.exec(x, y1)
        inv.exec(y1, y2)
    for _ in range(2):
        y1.zero_()
        y2.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(y1, ref1)
        assert torch.equal(y2, ref2)
    assert plan.status() == 0 and inv.status() == 0
    plan.destroy()
    inv.destroy()


@pytest.mark.parametrize("shape,batch", [((1 << 24,), 2), ((1 << 23,), 2), ((4096, 4096), 2)])
def test_two_column_kernels_batched(env, shape, batch):
    """The N = 4096 column passes (two columns per thread) over several
    transforms in one launch: the tile's transform index o enters the landing
    coordinates, the staged-store boxes (blocked output of the lifted pass 1,
    row blocks of the others) and the plain stores.  2^24 and 2^23 use them
    for both or the second lifted pass, 4096^2 for its column axis."""
    from paper_0811_2535_gb300 import inputs
    x = inputs.uniform((batch,) + shape, 6900 + len(shape) + batch)
    y, _ = run(env, list(shape), batch, -1, x)
    ref = oracle_ref(env, x, list(shape), batch, -1)
    assert per_transform_rel(y, ref, batch).max() <= TOL


@pytest.mark.parametrize("batch", [1, 2])
@pytest.mark.parametrize("sign", [-1, 1])
def test_3d_two_pass(env, batch, sign, monkeypatch):
    """256^3 in two passes (axis 1 lifted as 16 x 16): against the oracle,
    against one pass per axis (MOA_3D_TWO_PASS=0), and in place."""
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    monkeypatch.setenv("MOA_3D_TWO_PASS", "1")
    shape = (256, 256, 256)
    x = inputs.uniform((batch,) + shape, 6800 + batch)
    plan = moafft.Plan(list(shape), batch, sign)
    names = [plan.pass_info(i)["kernel"] for i in range(plan.info()["passes"])]
    plan.destroy()
    assert names == ["plane3d_p1_kernel", "pipe_col2_kernel<0,3>"], names
    y, _ = run(env, list(shape), batch, sign, x)
    yi, _ = run(env, list(shape), batch, sign, x, inplace=True)
    monkeypatch.setenv("MOA_3D_TWO_PASS", "0")
    y3, _ = run(env, list(shape), batch, sign, x)
    ref = oracle_ref(env, x, list(shape), batch, sign)
    assert per_transform_rel(y, ref, batch).max() <= TOL
    assert np.array_equal(y, yi)
    assert per_transform_rel(y3, ref, batch).max() <= TOL


@pytest.mark.parametrize("shape", [(1 << 24,), (4096, 4096), (256, 256, 256)])
def test_largest_plan(env, shape, monkeypatch):
    """The largest plan the library accepts: 127 transforms of 2^24 points
    (2^31 - 2^24 elements, 17 GB per buffer), so that element offsets above
    2^31 occur in every pass.  Transform b is the seeded full-size input rolled
    by 7919*b and scaled by 2^(b % 8 - 4) (exact in FP32).  Transforms 1 and 126
    are compared element by element with the oracle; every transform is checked
    by Parseval against its own input energy, which a transform written to a
    neighbour's place fails (the neighbours' scales differ by 2x)."""
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    monkeypatch.setenv("MOA_AUTOTUNE", "0")
    n, B = int(np.prod(shape)), 127
    base = inputs.uniform(shape, inputs.SEED_LARGE).reshape(-1)
    base_d = torch.from_numpy(base).cuda()
    x = torch.empty((B, n), dtype=torch.complex64, device="cuda")
    for b in range(B):
        x[b] = torch.roll(base_d, 7919 * b) * (2.0 ** (b % 8 - 4))
    plan = moafft.Plan(list(shape), B, -1)
    y = plan.exec(x)
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.destroy()
    for b in range(B):
        ex = float(torch.sum(torch.abs(x[b]).double() ** 2))
        ey = float(torch.sum(torch.abs(y[b]).double() ** 2))
        assert abs(ey / (n * ex) - 1.0) < 1e-5, (b, ey / (n * ex))
    for b in (1, B - 1):
        xb = (np.roll(base, 7919 * b) * np.float32(2.0 ** (b % 8 - 4))).astype(np.complex64)
        yb = y[b].cpu().numpy()
        ref = oracle_ref(env, xb, list(shape), 1, -1)
        assert per_transform_rel(yb, ref, 1).max() <= TOL, b
    del x, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("shape", [(1 << 20,), (4096, 4096), (256, 256, 256)])
def test_pipelined_wait_timeout_is_reported_and_contained(env, shape, monkeypatch):
    """Failure detection without a GPU fault: with MOA_FAULT_WAIT=1 at plan
    time the pipelined kernels give up on the first tile load that has not
    landed at its first test, wait for their loads in flight and return.  The
    plan's status word reads MOA_ERR_TIMEOUT (then clear), and a plan made
    afterwards on the same context is right."""
    torch, moafft, _ = env
    from paper_0811_2535_gb300 import inputs
    monkeypatch.setenv("MOA_AUTOTUNE", "0")
    x = inputs.uniform(shape, 4100)
    xd = torch.from_numpy(x.reshape(-1)).cuda()
    monkeypatch.setenv("MOA_FAULT_WAIT", "1")
    plan = moafft.Plan(list(shape), 1, -1)
    monkeypatch.delenv("MOA_FAULT_WAIT")
    assert any("pipe_col" in plan.pass_info(i)["kernel"] or "pipe_rowT" in plan.pass_info(i)["kernel"]
               for i in range(plan.info()["passes"]))
    plan.exec(xd)
    torch.cuda.synchronize()
    assert plan.status() == moafft.MOA_ERR_TIMEOUT
    assert plan.status() == 0
    plan.destroy()
    y, _ = run(env, list(shape), 1, -1, x)
    assert per_transform_rel(y, oracle_ref(env, x, list(shape), 1, -1), 1).max() <= TOL


@pytest.mark.parametrize("shape,batch,sign", [((1 << 25,), 1, -1), ((1 << 25,), 1, 1), ((1 << 26,), 1, -1),
                                              ((1 << 25,), 2, -1), ((8192, 2048), 1, -1), ((8192, 2048), 1, 1),
                                              ((2048, 8192), 1, -1), ((2048, 8192), 1, 1), ((16, 8192, 8), 2, 1),
                                              ((4, 4, 16384), 1, -1)])
def test_long_axes_against_oracle(env, shape, batch, sign):
    """1-D above 2^24 (three passes, n = r1*r2*c) and multi-D arrays with an
    axis above 4096 (that axis lifted L = L1*L2 inside the array, Eq. B.6):
    every element against the FP64 oracle."""
    from paper_0811_2535_gb300 import inputs
    n = 1
    for s_ in shape:
        n *= s_
    x = inputs.uniform((batch,) + tuple(shape), 7500 + len(shape) + batch + (n >> 20))
    y, info = run(env, list(shape), batch, sign, x)
    ref = oracle_ref(env, x, list(shape), batch, sign)
    assert per_transform_rel(y, ref, batch).max() <= TOL
    assert info["workspace_bytes"] == 8 * n * batch


@pytest.mark.parametrize("shape", [(1 << 25,), (8192, 2048), (2048, 8192)])
def test_long_axes_in_place(env, shape):
    """The first pass of a plan through the workspace keeps its tiles' places,
    so in == out is allowed."""
    from paper_0811_2535_gb300 import inputs
    x = inputs.uniform(shape, 7600 + len(shape))
    y, _ = run(env, list(shape), 1, -1, x, inplace=True)
    assert per_transform_rel(y, oracle_ref(env, x, list(shape), 1, -1), 1).max() <= TOL


def test_1d_2_28_closed_forms(env):
    """n = 2^28, where the oracle would take minutes: a shifted delta gives
    X[k] = w_n^(j0*k) (checked on 4096 sampled bins, exponent reduced exactly
    mod n in int64, FP64 reference), and Parseval holds on a random input."""
    torch, moafft, _ = env
    n = 1 << 28
    plan = moafft.Plan([n], 1, -1)
    assert plan.info()["passes"] == 3
    x = torch.zeros(n, dtype=torch.complex64, device="cuda")
    j0 = 123456789
    x[j0] = 1.0
    y = plan.exec(x)
    rng = np.random.default_rng(8)
    k = np.sort(rng.choice(n, 4096, replace=False)).astype(np.int64)
    got = y[torch.from_numpy(k).cuda()].cpu().numpy().astype(np.complex128)
    e = (j0 * k) % n
    ref = np.exp(-2j * np.pi * (e.astype(np.float64) / n))
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
    g = torch.Generator(device="cuda").manual_seed(9)
    xr = torch.complex(torch.rand(n, device="cuda", generator=g) * 2 - 1,
                       torch.rand(n, device="cuda", generator=g) * 2 - 1)
    yr = plan.exec(xr)
    assert plan.status() == 0
    ex = (xr.abs().double() ** 2).sum().item() * n
    ey = (yr.abs().double() ** 2).sum().item()
    assert abs(ey - ex) / ex <= 1e-6
    plan.destroy()
