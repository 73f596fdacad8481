"""Batched persistent launches against the FP64 oracle and the single-instance
kernels: uneven instance sizes (log-uniform, with empty and one-element
instances and misaligned slices), every batched op, and replay from a CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import (assert_dot, assert_normwise, assert_normwise_scaled, assert_reduced_sum,
                    assert_ulp, host)

pytestmark = pytest.mark.gpu


def lak():
    import paper_1409_0669_gb300 as m
    return m


def B():
    from paper_1409_0669_gb300 import batch
    return batch


def sizes(count, lo, hi, seed, extra=(0, 1, 2, 3)):
    s = list(synth.log_uniform_ints(count, lo, hi, seed))
    return list(extra) + s


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
def test_axpy_batch_vs_oracle(storage):
    """Every element of every instance against the oracle's y + alpha z rounded
    once to the storage type: bit-exact at alpha = 0.5 for FP32/FP64 (one
    rounding on both sides), within one ulp at alpha = -1.25 for FP32 (exact in
    the oracle's FP64) and for BF16/FP16 (the kernel rounds its FP32 result
    once more), within one FP64 rounding of each term for FP64 at -1.25.  Also
    identical bits to the single-instance vec_axpy."""
    ns = sizes(300, 1, 200_000, 1)
    dt = synth.torch_dtype(storage)
    ys = [synth.uniform(n + 1, 10 + i, storage).cuda()[1:] if i % 7 == 0 else
          synth.uniform(n, 10 + i, storage).cuda() for i, n in enumerate(ns)]
    zs = [synth.uniform(n, 5000 + i, storage).cuda() for i, n in enumerate(ns)]
    xs = [torch.empty(n, dtype=dt, device="cuda") for n in ns]
    alphas = [0.5 if i % 2 else -1.25 for i in range(len(ns))]
    b = B().axpy_batch(xs, ys, zs, alphas)
    b.run()
    torch.cuda.synchronize()
    for i, (x, y, z, a) in enumerate(zip(xs, ys, zs, alphas)):
        ref64 = oracle.axpy(y.cpu(), z.cpu(), a)
        ref = oracle.round_to(ref64, storage)
        got = host(x)
        if a == 0.5 and storage in ("f32", "f64"):
            assert np.array_equal(got, ref), f"instance {i} (n={ns[i]}): alpha = 0.5 bit-exact"
        elif storage == "f64":
            # the oracle's own alpha * z is rounded in FP64 (the kernel fuses it):
            # one rounding of each of |y + alpha z| and |alpha z| apart
            bound = 2.0 ** -52 * (np.abs(ref64) + np.abs(a * host(z)))
            assert np.all(np.abs(got - ref64) <= bound), f"instance {i} (n={ns[i]})"
        else:
            assert_ulp(got, ref, storage, 1.0, f"instance {i} (n={ns[i]})")
        single = torch.empty_like(x)
        lak().vec_axpy(single, y, z, a)
        torch.cuda.synchronize()
        assert torch.equal(x, single)


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
def test_dot_batch_vs_oracle(storage):
    ns = sizes(400, 1, 300_000, 2)
    xs = [synth.uniform(n, 20 + i, storage).cuda() for i, n in enumerate(ns)]
    ys = [synth.uniform(n, 9000 + i, storage).cuda() for i, n in enumerate(ns)]
    odt = torch.float64 if storage == "f64" else torch.float32
    out = torch.full((len(ns),), float("nan"), dtype=odt, device="cuda")
    outs = [out[i:i + 1] for i in range(len(ns))]
    b = B().dot_batch(xs, ys, outs)
    for rep in range(3):                    # the arrival counters are reused
        b.run()
        torch.cuda.synchronize()
        got = out.cpu().double().numpy()
        for i, (x, y) in enumerate(zip(xs, ys)):
            assert_dot(got[i], oracle.dot(x.cpu(), y.cpu()), host(x), host(y), storage,
                       f"instance {i} (n={ns[i]}) rep {rep}")
    assert torch.all(b.workspace[:65536] == 0)


@pytest.mark.parametrize("cfg", [None, (64, 0, 8, 0), (128, 0, 2, 0)], ids=str)
@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
def test_gemv_batch_vs_oracle(storage, cfg):
    """Instances of 1..700 rows and columns with padded leading dimensions:
    rows go 1..4 at a time per lane group depending on the row length and the
    access width (several rows a stride apart that share their alignment)."""
    ms = sizes(80, 1, 700, 3, extra=(1, 5, 0))
    ns = sizes(80, 1, 700, 4, extra=(1, 0, 9))
    dt = synth.torch_dtype(storage)
    As, xs, ys, fulls = [], [], [], []
    for i, (m, n) in enumerate(zip(ms, ns)):
        pad = 3 if i % 5 == 0 else 0
        full = synth.normal((m, n + pad), 30 + i, storage).cuda()
        fulls.append(full)
        As.append(full[:, :n])
        xs.append(synth.uniform(n, 40 + i, storage).cuda())
        ys.append(torch.full((m,), float("nan"), dtype=dt, device="cuda"))
    b = B().gemv_batch(As, xs, ys, cfg=cfg)
    b.run()
    torch.cuda.synchronize()
    for i, (A, x, y) in enumerate(zip(As, xs, ys)):
        m, n = A.shape
        if m == 0:
            continue
        if n == 0:
            assert torch.all(y == 0)
            continue
        lda = fulls[i].shape[1]
        flat = fulls[i].reshape(-1).cpu()
        ref = oracle.gemv(flat, x.cpu(), m, n, lda, "row")
        abs_ref = oracle.gemv(np.nan_to_num(np.abs(oracle.widen(flat))), np.abs(host(x)), m, n,
                              lda, "row")
        if storage in ("bf16", "f16"):          # FP32 sums rounded once to the storage
            assert_reduced_sum(host(y), ref, abs_ref, np.full(m, n), storage,
                               f"instance {i} {m}x{n}")
        else:
            assert_normwise_scaled(host(y), ref, abs_ref, storage, f"instance {i} {m}x{n}")


@pytest.mark.parametrize("cfg", [None, (128, 0, 8, 0), (128, 0, 4, 0)])
@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
def test_gemv_batch_long_rows_vs_oracle(storage, cfg):
    """Rows long enough for the plan to give them whole warps (several warps per
    row, added in warp order through shared memory), with padded leading
    dimensions and odd lengths, next to short rows in the same batch."""
    ms = sizes(18, 1, 300, 7, extra=(1, 3, 64))
    ns = sizes(18, 1000, 6000, 8, extra=(2048, 2049, 4099, 8192))
    dt = synth.torch_dtype(storage)
    As, xs, ys, fulls = [], [], [], []
    for i, (m, n) in enumerate(zip(ms, ns)):
        m, n = int(m), int(n)
        pad = 5 if i % 3 == 0 else 0
        full = synth.normal((m, n + pad), 90 + i, storage).cuda()
        fulls.append(full)
        As.append(full[:, :n])
        xs.append(synth.uniform(n, 190 + i, storage).cuda())
        ys.append(torch.full((m,), float("nan"), dtype=dt, device="cuda"))
    b = B().gemv_batch(As, xs, ys, cfg=cfg)
    b.run()
    torch.cuda.synchronize()
    for i, (A, x, y) in enumerate(zip(As, xs, ys)):
        m, n = A.shape
        lda = fulls[i].shape[1]
        flat = fulls[i].reshape(-1).cpu()
        ref = oracle.gemv(flat, x.cpu(), m, n, lda, "row")
        abs_ref = oracle.gemv(np.nan_to_num(np.abs(oracle.widen(flat))), np.abs(host(x)), m, n,
                              lda, "row")
        if storage in ("bf16", "f16"):          # FP32 sums rounded once to the storage
            assert_reduced_sum(host(y), ref, abs_ref, np.full(m, n), storage,
                               f"instance {i} {m}x{n}")
        else:
            assert_normwise_scaled(host(y), ref, abs_ref, storage, f"instance {i} {m}x{n}")


@pytest.mark.parametrize("cfg", [None, (32, 0, 4, 0), (128, 0, 8, 0), (512, 0, 4, 0)])
@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
def test_spmv_batch_vs_oracle(storage, cfg):
    """Every launch shape maps tickets to (unit, warp slot) with its own warps
    per block: one warp (32), four (128, 8 entries per lane) and sixteen (512)."""
    csrs, xs, ys, refs, bars = [], [], [], [], []
    rows = sizes(24, 1000, 20_000, 5, extra=(1, 31, 33))
    for i, m in enumerate(rows):
        if i == 3:
            rp, ci, v = synth.laplacian_2d(64, storage)
            m = 64 * 64
        elif i == 4:
            rp, ci, v = synth.random_csr(m, m, 60 + i, storage, 0, 40, 0.3)
        else:
            rp, ci, v = synth.banded_random_csr(m, 60 + i, 5, 64, storage)
        x = synth.uniform(m, 70 + i, storage)
        csrs.append((rp.cuda(), ci.cuda(), v.cuda(), m))
        xs.append(x.cuda())
        ys.append(torch.full((m,), float("nan"), dtype=v.dtype, device="cuda"))
        refs.append(oracle.csr_spmv(rp, ci, v, x))
        bars.append((oracle.csr_spmv(rp, ci, np.abs(oracle.widen(v)), np.abs(oracle.widen(x))),
                     np.diff(rp.numpy()).astype(np.float64)))
    b = B().spmv_batch(csrs, xs, ys, cfg=cfg)
    b.run()
    torch.cuda.synchronize()
    for i, (y, r) in enumerate(zip(ys, refs)):
        if storage in ("bf16", "f16"):          # FP32 sums rounded once to the storage
            assert_reduced_sum(host(y), r, bars[i][0], bars[i][1], storage, f"instance {i}")
        else:
            assert_normwise(host(y), r, storage, f"instance {i}")


def test_batch_replays_from_cuda_graph():
    ns = sizes(64, 100, 50_000, 6)
    xs = [synth.uniform(n, 80 + i, "f32").cuda() for i, n in enumerate(ns)]
    ys = [synth.uniform(n, 180 + i, "f32").cuda() for i, n in enumerate(ns)]
    out = torch.zeros(len(ns), device="cuda")
    b = B().dot_batch(xs, ys, [out[i:i + 1] for i in range(len(ns))])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(s)                              # warm: loads the kernels before capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    first = out.clone()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run()
    for _ in range(5):
        out.zero_()
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, first)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_families_back_to_back_in_one_graph(storage):
    """The dot, GEMV and CSR batches captured back to back in one graph (each
    kernel waits for the one before; the GEMV lets the next launch only when it
    has finished): outputs identical to the same batches run one at a time,
    over several replays that each start from overwritten outputs."""
    dt = synth.torch_dtype(storage)
    ns = sizes(40, 100, 20_000, 9)
    xs = [synth.uniform(n, 300 + i, storage).cuda() for i, n in enumerate(ns)]
    zs = [synth.uniform(n, 400 + i, storage).cuda() for i, n in enumerate(ns)]
    dots = torch.zeros(len(ns), device="cuda")
    shapes = list(zip(sizes(30, 1, 600, 10, extra=(1, 4)), sizes(30, 1, 900, 11, extra=(7, 64))))
    As = [synth.normal((m, n), 500 + i, storage).cuda() for i, (m, n) in enumerate(shapes)]
    gx = [synth.uniform(n, 600 + i, storage).cuda() for i, (m, n) in enumerate(shapes)]
    gy = [torch.zeros(m, dtype=dt, device="cuda") for m, _ in shapes]
    csrs, cx, cy = [], [], []
    for i, m in enumerate(sizes(12, 500, 20_000, 12)):
        rp, ci, v = synth.random_csr(m, m, 700 + i, storage, min_len=5, max_len=64)
        csrs.append((rp.cuda(), ci.cuda(), v.cuda(), m))
        cx.append(synth.uniform(m, 800 + i, storage).cuda())
        cy.append(torch.zeros(m, dtype=dt, device="cuda"))
    bd = B().dot_batch(xs, zs, [dots[i:i + 1] for i in range(len(ns))])
    bg = B().gemv_batch(As, gx, gy)
    bs = B().spmv_batch(csrs, cx, cy)
    outs = [dots] + gy + cy
    for b in (bd, bg, bs):
        b.run()
    torch.cuda.synchronize()
    alone = [o.clone() for o in outs]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for b in (bd, bg, bs):
            b.run(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for b in (bd, bg, bs):
            b.run()
    for _ in range(3):
        for o in outs:
            o.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for o, a in zip(outs, alone):
            assert torch.equal(o, a)


def test_spmv_batch_ticket_counters_reset_between_runs():
    """The CSR batch's warps take their rows from ticket counters in the
    workspace, which the last warp resets: every run, direct or replayed from a
    CUDA graph, must compute the product for the inputs it finds, and the
    counter area must be zero again afterwards."""
    csrs, xs, ys, hosts = [], [], [], []
    for i, m in enumerate([1, 33, 4000, 20_000, 65]):
        rp, ci, v = synth.banded_random_csr(m, 300 + i, 5, 64, "f32")
        csrs.append((rp.cuda(), ci.cuda(), v.cuda(), m))
        hosts.append((rp, ci, v))
        xs.append(torch.empty(m, device="cuda"))
        ys.append(torch.full((m,), float("nan"), device="cuda"))
    b = B().spmv_batch(csrs, xs, ys)

    def check(seed):
        torch.cuda.synchronize()
        for i, ((rp, ci, v), y) in enumerate(zip(hosts, ys)):
            x = synth.uniform(rp.numel() - 1, seed + i, "f32")
            assert_normwise(host(y), oracle.csr_spmv(rp, ci, v, x), "f32", f"instance {i}")
        assert int(b.workspace[:16].count_nonzero()) == 0

    def load(seed):
        for i, x in enumerate(xs):
            x.copy_(synth.uniform(x.numel(), seed + i, "f32").cuda())
            ys[i].fill_(float("nan"))

    for rep in range(3):
        load(400 + 10 * rep)
        b.run()
        check(400 + 10 * rep)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.run(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run()
    for rep in range(3):
        load(500 + 10 * rep)
        g.replay()
        check(500 + 10 * rep)


def test_batching_workload_sampled_instances_vs_oracle():
    """The batching workload itself, at its full size: 4096 uneven FP32
    instances per family (vectors of 256..1M entries, GEMVs of 64..4096 rows
    and columns, CSR blocks of 1k..200k rows with 5..64 entries per row), each
    family in one persistent launch with the default launch shapes.  At least
    64 instances per family (the smallest, the largest and a seeded random
    choice) are checked element by element against the oracle."""
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = synth.batch_workload(dev, 4096, 4000)
    count = 4096
    pick = set(synth.rng(4100).choice(count, 62, replace=False).tolist())

    def chosen(sizes_):
        return sorted(pick | {int(np.argmin(sizes_)), int(np.argmax(sizes_))})

    ys = [v[0] for v in wl["vec"]]
    zs = [v[1] for v in wl["vec"]]
    xs = [v[2] for v in wl["vec"]]
    outs = torch.full((count,), float("nan"), device=dev)
    bx = B().axpy_batch(xs, ys, zs, [0.5] * count)
    bd = B().dot_batch(ys, zs, [outs[i:i + 1] for i in range(count)])
    bx.run()
    bd.run()
    torch.cuda.synchronize()
    sel = chosen([y.numel() for y in ys])
    assert len(sel) >= 64
    dots = outs.cpu().double().numpy()
    for i in sel:
        yc, zc = ys[i].cpu(), zs[i].cpu()
        ref = oracle.round_to(oracle.axpy(yc, zc, 0.5), "f32")
        assert np.array_equal(host(xs[i]), ref), f"axpy instance {i}"
        assert_dot(dots[i], oracle.dot(yc, zc), host(ys[i]), host(zs[i]), "f32",
                   f"dot instance {i}")
    del bx, bd

    As = [g[0] for g in wl["gemv"]]
    bg = B().gemv_batch(As, [g[1] for g in wl["gemv"]], [g[2] for g in wl["gemv"]])
    bg.run()
    torch.cuda.synchronize()
    sel = chosen([A.numel() for A in As])
    assert len(sel) >= 64
    for i in sel:
        A, x, y = wl["gemv"][i]
        m, n = A.shape
        flat = A.reshape(-1).cpu()
        ref = oracle.gemv(flat, x.cpu(), m, n, n, "row")
        abs_ref = oracle.gemv(np.abs(oracle.widen(flat)), np.abs(host(x)), m, n, n, "row")
        assert_normwise_scaled(host(y), ref, abs_ref, "f32", f"gemv instance {i} {m}x{n}")
    del bg

    bs = B().spmv_batch([c[0] for c in wl["csr"]], [c[1] for c in wl["csr"]],
                        [c[2] for c in wl["csr"]])
    bs.run()
    torch.cuda.synchronize()
    sel = chosen([c[0][3] for c in wl["csr"]])
    assert len(sel) >= 64
    for i in sel:
        (rp, ci, v, m), x, y = wl["csr"][i]
        ref = oracle.csr_spmv(rp.cpu(), ci.cpu(), v.cpu(), x.cpu())
        assert_normwise(host(y), ref, "f32", f"spmv instance {i} ({m} rows)")
    assert int(bs.workspace[:16].count_nonzero()) == 0


def test_batches_take_the_shipped_tuned_defaults():
    """A batch planned without a cfg on a GPU that the shipped autotuner cache
    covers takes the cached launch shape (the built-in table is only the
    fallback)."""
    import json

    from paper_1409_0669_gb300 import autotune
    key = autotune.cache_key()
    with open(B().TUNED_DEFAULTS) as fh:
        entries = json.load(fh).get(key)
    if not entries:
        pytest.skip(f"no shipped batched defaults for {key}")
    for name, cfg in entries.items():
        _, op, storage = name.split(":")
        dt = synth.torch_dtype(storage)
        n = 1000
        v = [torch.ones(n, dtype=dt, device="cuda")]
        if op == "axpy":
            b = B().axpy_batch(v, v, v, [0.5])
        elif op == "dot":
            b = B().dot_batch(v, v, [torch.zeros(1, dtype=torch.float64 if storage == "f64"
                                                 else torch.float32, device="cuda")])
        elif op == "gemv_row":
            b = B().gemv_batch([torch.ones(4, n, dtype=dt, device="cuda")], v,
                               [torch.zeros(4, dtype=dt, device="cuda")])
        else:
            rp, ci, vals = synth.laplacian_2d(8, storage)
            b = B().spmv_batch([(rp.cuda(), ci.cuda(), vals.cuda(), 64)],
                               [torch.ones(64, dtype=dt, device="cuda")],
                               [torch.zeros(64, dtype=dt, device="cuda")])
        assert tuple(b.info.cfg.as_tuple()) == tuple(cfg), (name, b.info.cfg.as_tuple(), cfg)


@pytest.mark.parametrize("vec", [2, 4, 8, 16])
@pytest.mark.parametrize("storage", ["f32", "f64", "bf16"])
def test_gemv_batch_adversarial_shapes(storage, vec):
    """Row counts below and around the rows a lane group takes at once, row
    lengths around the access width and the lane-group thresholds, leading
    dimensions that give every alignment period, and matrices starting 0..3
    elements past an aligned address: every instance against the oracle."""
    dt = synth.torch_dtype(storage)
    ms = (1, 2, 3, 4, 5, 7, 8, 9, 17, 33)
    ns = (1, 2, 3, 5, 8, 9, 31, 33, 64, 65, 129, 257, 513, 1025)
    shapes = [(m, n, pad, off) for i, (m, n) in enumerate((m, n) for m in ms for n in ns)
              for pad, off in [((i * 7) % 4, (i * 5) % 4)]]
    total = sum(off + m * (n + pad) for m, n, pad, off in shapes) + 64
    flat = synth.normal((total,), 600, storage).cuda()
    As, xs, ys, metas = [], [], [], []
    o = 0
    for i, (m, n, pad, off) in enumerate(shapes):
        o += off
        A = flat[o:o + m * (n + pad)].view(m, n + pad)[:, :n]
        o += m * (n + pad)
        As.append(A)
        xs.append(synth.uniform(n, 700 + i, storage).cuda())
        ys.append(torch.full((m,), float("nan"), dtype=dt, device="cuda"))
        metas.append((m, n, n + pad))
    b = B().gemv_batch(As, xs, ys, cfg=(128, 0, vec, 0))
    b.run()
    torch.cuda.synchronize()
    for i, (A, x, y, (m, n, lda)) in enumerate(zip(As, xs, ys, metas)):
        sub = A.contiguous().reshape(-1).cpu()              # the instance's own entries
        ref = oracle.gemv(sub, x.cpu(), m, n, n, "row")
        abs_ref = oracle.gemv(np.abs(oracle.widen(sub)), np.abs(host(x)), m, n, n, "row")
        what = f"instance {i} {m}x{n} lda {lda} vec {vec}"
        if storage == "bf16":
            assert_reduced_sum(host(y), ref, abs_ref, np.full(m, n), storage, what)
        else:
            assert_normwise_scaled(host(y), ref, abs_ref, storage, what)


@pytest.mark.parametrize("vec", [4, 8, 16])
@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
def test_gemv_batch_misaligned_x(storage, vec):
    """Right-hand sides that start 0..7 elements past an aligned address (views
    of one buffer), against matrices whose rows start at every offset: the x
    reads of the shared-memory ring path and of the register path, aligned and
    element by element, every instance against the oracle."""
    dt = synth.torch_dtype(storage)
    shapes = [(m, n) for m in (1, 4, 5, 9, 33) for n in (7, 16, 31, 64, 100, 257, 1000)]
    xtotal = sum(n + 8 for _, n in shapes)
    xflat = synth.uniform(xtotal, 800, storage).cuda()
    As, xs, ys = [], [], []
    xo = 0
    for i, (m, n) in enumerate(shapes):
        lda = n + i % 3
        As.append(synth.normal((m * lda,), 900 + i, storage).cuda().view(m, lda)[:, :n])
        off = i % 8
        xs.append(xflat[xo + off:xo + off + n])
        xo += n + 8
        ys.append(torch.full((m,), float("nan"), dtype=dt, device="cuda"))
    b = B().gemv_batch(As, xs, ys, cfg=(128, 0, vec, 0))
    b.run()
    torch.cuda.synchronize()
    for i, (A, x, y, (m, n)) in enumerate(zip(As, xs, ys, shapes)):
        sub = A.contiguous().reshape(-1).cpu()
        ref = oracle.gemv(sub, x.cpu(), m, n, n, "row")
        abs_ref = oracle.gemv(np.abs(oracle.widen(sub)), np.abs(host(x)), m, n, n, "row")
        what = f"instance {i} {m}x{n} x offset {i % 8} vec {vec}"
        if storage in ("bf16", "f16"):
            assert_reduced_sum(host(y), ref, abs_ref, np.full(m, n), storage, what)
        else:
            assert_normwise_scaled(host(y), ref, abs_ref, storage, what)
