"""CUDA path vs the FP64 oracle, element by element (relative L2 over all
stored entries): <= 1e-13 for FP64 and <= 5e-6 for FP32, on seeded inputs.

Sizes cover every compiled line length on each axis (several tiles and a
ragged tail where the tile width does not divide the column count), both
layouts (out-of-place dense, in-place padded), and the degenerate lengths 1
and 2.  Runs on a GPU only."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, gpu_c2r, gpu_r2c, np_round, rel_l2

pytestmark = pytest.mark.gpu

COL_LENGTHS = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048,
               3, 6, 12, 24, 48, 96, 192, 384, 768, 1536]
Z_HALF = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 3, 6, 12, 24, 48, 96, 192, 384, 768]

SHAPES = sorted(set(
    [(L, 6, 8) for L in COL_LENGTHS]
    + [(4, L, 12) for L in COL_LENGTHS]
    + [(3, 4, 2 * M) for M in Z_HALF]
    + [(1, 1, 2), (2, 2, 2), (1, 4, 8), (4, 1, 8), (16, 16, 16), (24, 48, 96)]
    + [(3, 1, 1024), (1, 1, 1024), (3, 3, 1024)]  # odd line counts: FP64 lines of 1024 points run in pairs
))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2202_12756_gb300 as fft3d
    fft3d.load_library()


def check_pair(shape, name, inplace, seed=0):
    f = np_round(synth.uniform_field(shape, seed), name)
    F_ref = oracle.rfft3(f)
    F = gpu_r2c(f, name, inplace)
    assert not np.isnan(F).any(), "unwritten output entries"
    e1 = rel_l2(F, F_ref)
    assert e1 <= TOL[name], (shape, name, inplace, "r2c", e1)
    G = synth.random_half_spectrum(shape, seed + 100)
    if name == "f32":
        G = G.astype(np.complex64).astype(np.complex128)
    g_ref = oracle.irfft3(G, shape)
    g = gpu_c2r(G, shape, name, inplace)
    assert not np.isnan(g).any(), "unwritten output entries"
    e2 = rel_l2(g, g_ref)
    assert e2 <= TOL[name], (shape, name, inplace, "c2r", e2)
    return e1, e2


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", ["f64", "f32"])
def test_parity_sweep_out_of_place(shape, name):
    check_pair(shape, name, inplace=False)


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 4, 6), (64, 32, 48), (2048, 6, 8), (4, 1536, 12), (3, 4, 2048)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", ["f64", "f32"])
def test_parity_in_place(shape, name):
    check_pair(shape, name, inplace=True)


@pytest.mark.parametrize("name", ["f64", "f32"])
def test_config_64cubed(name):
    """64^3, iid uniform[-1, 1) from seed 0, out-of-place and in-place."""
    shape = (64, 64, 64)
    f = np_round(synth.uniform_field(shape, 0), name)
    F_ref = oracle.rfft3(f)
    for inplace in (False, True):
        F = gpu_r2c(f, name, inplace)
        assert rel_l2(F, F_ref) <= TOL[name]
        back = gpu_c2r(F_ref, shape, name, inplace)
        assert rel_l2(back, f) <= TOL[name]


def test_layouts_agree_bitwise():
    shape = (32, 48, 64)
    f = synth.uniform_field(shape, 3)
    for name in ("f64", "f32"):
        a = gpu_r2c(f, name, inplace=False)
        b = gpu_r2c(f, name, inplace=True)
        assert np.array_equal(a, b)
        G = oracle.rfft3(f)
        assert np.array_equal(gpu_c2r(G, shape, name, False), gpu_c2r(G, shape, name, True))


def test_out_of_place_preserves_input():
    import torch
    import paper_2202_12756_gb300 as fft3d
    shape = (24, 32, 48)
    plan = fft3d.get_plan(shape, torch.float64, "cuda")
    x = torch.from_numpy(synth.uniform_field(shape, 4)).cuda()
    x0 = x.clone()
    X = plan.r2c(x)
    X0 = X.clone()
    plan.c2r(X)
    torch.cuda.synchronize()
    assert torch.equal(x, x0)
    assert torch.equal(X, X0)


def test_eq5_field_closed_form_and_round_trip():
    """Eq. 5 field: exact spectrum i (+-1) N^3 at (+-1, +-2, 3), (+-4, +-5, 6) and
    the double-precision round trip at the 1e-14 level stated in Sec. 4."""
    n = 64
    f = synth.eq5_field(n, n, n)
    F = gpu_r2c(f, "f64")
    ref = np.zeros_like(F)
    for (a0, a1, a2) in ((1, 2, 3), (4, 5, 6)):
        for s0 in (1, -1):
            for s1 in (1, -1):
                ref[(s0 * a0) % n, (s1 * a1) % n, a2] = 1j * s0 * s1 * n ** 3
    assert np.max(np.abs(F - ref)) < 1e-9 * n ** 3
    back = gpu_c2r(F, (n, n, n), "f64")
    assert np.max(np.abs(back - f)) / np.max(np.abs(f)) < 1e-14


def test_plane_waves_512_fp64():
    """512^3 FP64: uniform noise + 8 seeded plane waves, |k_i| < 256, seed 1.
    Full oracle parity, and the wave part against its closed form."""
    from oracle_pins import plane_wave_spectrum
    shape = (512, 512, 512)
    noise = synth.uniform_field(shape, 1)
    kv = synth.plane_wave_vectors(1, count=8, kmax=256)
    waves = synth.plane_waves(shape, kv)
    f = noise + waves
    F = gpu_r2c(f, "f64")
    F_ref = oracle.rfft3(f)
    assert rel_l2(F, F_ref) <= TOL["f64"]
    F_noise = gpu_r2c(noise, "f64")
    W = plane_wave_spectrum(shape, kv)
    assert np.max(np.abs((F - F_noise) - W)) < 1e-9 * np.prod(shape)
    back = gpu_c2r(F, shape, "f64")
    assert rel_l2(back, f) <= TOL["f64"]


FUSED_SHAPES = [(4, 512, 512), (2, 1024, 1024), (3, 768, 768), (2, 1536, 1536), (1, 2048, 2048),
                (6, 1024, 1024)]


@pytest.mark.parametrize("shape", FUSED_SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_fused_plane_pass_parity(shape):
    """Float plans with (N1, N2) in the fused set can run axes 2 and 1 as one
    persistent kernel (planes handed over through L2); same results bar."""
    import torch
    import paper_2202_12756_gb300 as fft3d
    plan = fft3d.get_plan(shape, torch.float32, "cuda")
    plan.set_fused(True)
    try:
        assert plan.info()["fused_plane_pass"]
        for inplace in (False, True):
            check_pair(shape, "f32", inplace, seed=7)
        assert plan.status() == 0
    finally:
        plan.set_fused(False)


def test_fused_plane_pass_not_offered_elsewhere():
    import torch
    import paper_2202_12756_gb300 as fft3d
    for shape, dt in (((8, 256, 256), torch.float32), ((4, 512, 512), torch.float64), ((4, 512, 256), torch.float32)):
        plan = fft3d.Plan(shape, dt)
        with pytest.raises(fft3d.FFT3DError) as e:
            plan.set_fused(True)
        assert e.value.status == fft3d.FFT3D_ERR_SIZE
        assert not plan.info()["fused_plane_pass"]


@pytest.mark.parametrize("shape", [(16, 24, 32), (64, 32, 48), (1, 4, 8), (8, 1024, 12)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", ["f64", "f32"])
def test_c2r_overwrite(shape, name):
    """Inverse that uses its input as work space: same result as the
    input-preserving inverse; the dense output is written by the last pass."""
    import torch
    import paper_2202_12756_gb300 as fft3d
    from gpu_util import torch_dtype
    dt = torch_dtype(name)
    plan = fft3d.get_plan(shape, dt, "cuda")
    G = synth.random_half_spectrum(shape, 71)
    if name == "f32":
        G = G.astype(np.complex64).astype(np.complex128)
    X = torch.from_numpy(G).to(fft3d.complex_of(dt)).cuda()
    out = torch.full(shape, float("nan"), dtype=dt, device="cuda")
    plan.c2r_overwrite(X, out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), oracle.irfft3(G, shape)) <= TOL[name]


@pytest.mark.parametrize("shape", [(32, 64, 128), (64, 256, 256), (16, 256, 1024)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", ["f64", "f32"])
def test_host_resident_field(name, shape):
    """Forward from, and overwrite-inverse into, pinned host memory (read and
    written directly by the first and last passes, which then run on a
    limited grid of blocks looping over the lines when there are more line
    groups than that: 512 groups at 64 x 256 x 256, and at 16 x 256 x 1024,
    where FP64 lines run two per complex transform).  Same arithmetic as the
    device-resident calls, so the results must agree bit for bit."""
    import torch
    import paper_2202_12756_gb300 as fft3d
    from gpu_util import torch_dtype
    dt = torch_dtype(name)
    plan = fft3d.get_plan(shape, dt, "cuda")
    f = np_round(synth.uniform_field(shape, 72), name)
    host_in = torch.from_numpy(f).to(dt).pin_memory()
    host_out = torch.full(shape, float("nan"), dtype=dt).pin_memory()
    X = plan.r2c(host_in)
    X_dev = plan.r2c(host_in.cuda())
    torch.cuda.synchronize()
    assert torch.equal(X, X_dev)
    assert rel_l2(X.cpu().numpy(), oracle.rfft3(f)) <= TOL[name]
    y_dev = plan.c2r_overwrite(X_dev)
    plan.c2r_overwrite(X, host_out)
    torch.cuda.synchronize()
    assert torch.equal(host_out, y_dev.cpu())
    assert rel_l2(host_out.numpy(), f) <= TOL[name]


@pytest.mark.parametrize("shape", [(4, 1024, 64), (6, 2048, 64), (1024, 16, 32), (2048, 16, 32), (1024, 1024, 32)],
                         ids=lambda s: "x".join(map(str, s)))
def test_tma_staged_column_passes(shape):
    """Float column passes of 1024 / 2048 points stage full tiles with TMA
    tensor copies: one map over aligned rows (x-pass), or even / odd row maps
    when the y-pass row pitch (N2/2 + 1 complex) is odd.  Both layouts."""
    for inplace in (False, True):
        check_pair(shape, "f32", inplace, seed=9)


@pytest.mark.parametrize("shape", [(1536, 16, 32), (1536, 24, 24), (6, 1536, 64), (4, 1536, 96), (1536, 1536, 32)],
                         ids=lambda s: "x".join(map(str, s)))
def test_one_buffer_pipelined_column_passes(shape):
    """The float x-pass of 1536 points runs on the persistent kernel whose
    staging buffer is also the transform's exchange buffer: tiles staged by
    TMA (1536 x 16 x 32: 16 * 17 = 272 columns, 17 full tiles; 1536 x 1536 x
    32 with the one-tile y-pass of the same length) or per element with a
    ragged last tile (24 * 13 = 312 columns).  The 1536-point y-passes of
    (6, 1536, 64) and (4, 1536, 96) stay on the one-tile kernel.  Both
    directions, element by element against the oracle."""
    for inplace in (False, True):
        check_pair(shape, "f32", inplace, seed=23)


@pytest.mark.parametrize("shape", [(2048, 64, 64), (2048, 24, 24), (32, 2048, 64), (3, 2048, 192)],
                         ids=lambda s: "x".join(map(str, s)))
def test_cta_pair_column_passes(shape):
    """Float columns of 2048 points run on clusters of two CTAs, each holding
    one row parity of a 16-column tile (1024-point FFTs, then one radix-2
    step across the pair through distributed shared memory).  Shapes: x-pass
    tiles staged by TMA from the row-pair map (2048 x 64 x 64: 64 * 33
    columns, 132 full tiles), per-element copies with a ragged last tile
    (24 * 13 = 312 columns), y-pass even / odd row maps (in place, odd pitch
    33 or 97) or the row-pair map over the split layout (out of place); both
    directions, element by element against the oracle."""
    for inplace in (False, True):
        check_pair(shape, "f32", inplace, seed=17)


@pytest.mark.parametrize("name", ["f64", "f32"])
def test_cuda_graph_capture_and_replay(name):
    """The exec calls only enqueue work on the caller's stream, so a forward +
    inverse pair can be captured once into a CUDA graph and replayed (the way
    to remove launch gaps for small transforms); replays must reproduce the
    eager results bit for bit."""
    import torch
    import paper_2202_12756_gb300 as fft3d
    from gpu_util import torch_dtype
    dt = torch_dtype(name)
    shape = (32, 48, 64)
    plan = fft3d.get_plan(shape, dt, "cuda")
    f = np_round(synth.uniform_field(shape, 95), name)
    x = torch.from_numpy(f).to(dt).cuda()
    X_eager = plan.r2c(x)
    y_eager = plan.c2r(X_eager)
    X = plan.empty_complex()
    y = plan.empty_real()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside the capture
        plan.r2c(x, X)
        plan.c2r(X, y)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    X.zero_()
    y.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.r2c(x, X)
        plan.c2r(X, y)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(X, X_eager)
    assert torch.equal(y, y_eager)
    assert rel_l2(y.cpu().numpy(), f) <= TOL[name]
