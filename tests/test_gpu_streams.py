"""Several streams transforming at the same time.

A plan serves one stream at a time: the out-of-place inverse keeps the
k2 = N2/2 column in the plan's scratch plane, and the pipelined column passes
draw their tiles from the plan's tile counter.  The binding therefore caches
one plan per (shape, dtype, device, batch, stream).  Here irfft3 and rfft3 run
on two streams at once, several times each, and every result must match the
FP64 oracle element by element."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,shape", [("f64", (128, 256, 256)), ("f32", (1024, 32, 64))],
                         ids=["f64-128x256x256", "f32-1024x32x64"])
def test_two_streams_at_once(name, shape):
    import torch
    import paper_2202_12756_gb300 as fft3d
    dt = torch.float32 if name == "f32" else torch.float64
    cdt = fft3d.complex_of(dt)
    Gs, fs = [], []
    for i in range(2):
        G = synth.random_half_spectrum(shape, 50 + i)
        f = synth.uniform_field(shape, 60 + i)
        if name == "f32":
            G = G.astype(np.complex64).astype(np.complex128)
            f = f.astype(np.float32).astype(np.float64)
        Gs.append(G)
        fs.append(f)
    g_refs = [oracle.irfft3(G, shape) for G in Gs]
    F_refs = [oracle.rfft3(f) for f in fs]
    Xs = [torch.from_numpy(G).to(cdt).cuda() for G in Gs]
    xs = [torch.from_numpy(f).to(dt).cuda() for f in fs]
    streams = [torch.cuda.Stream() for _ in range(2)]
    torch.cuda.synchronize()
    outs = [[], []]
    for _ in range(4):
        for i in range(2):
            with torch.cuda.stream(streams[i]):
                outs[i].append((fft3d.irfft3(Xs[i], shape), fft3d.rfft3(xs[i])))
    torch.cuda.synchronize()
    for i in range(2):
        for g, F in outs[i]:
            assert rel_l2(g.cpu().numpy(), g_refs[i]) <= TOL[name]
            assert rel_l2(F.cpu().numpy(), F_refs[i]) <= TOL[name]


@pytest.mark.parametrize("shape", [(1024, 64, 64), (64, 1024, 64)], ids=lambda s: "x".join(map(str, s)))
def test_fields_in_flight_through_copy_engines(shape):
    """The end-to-end pattern the bench times: three fields in flight, each
    on its own stream with its own plan, copied from page-locked host memory
    (anonymous memory registered with cudaHostRegister) into a dense device
    array, transformed forward out of place, taken back with the overwriting
    inverse, and copied out.  Every field's spectrum must match the FP64
    oracle, and every result must equal, bit for bit, the same calls made on
    one stream one field at a time."""
    import torch
    import bench
    import paper_2202_12756_gb300 as fft3d
    nf = 3
    fs = [synth.uniform_field(shape, 80 + i).astype(np.float32) for i in range(nf)]
    F_refs = [oracle.rfft3(f.astype(np.float64)) for f in fs]
    hb = bench.HostBuffers()
    try:
        host_in = [hb.empty(shape) for _ in range(nf)]
        host_out = [hb.empty(shape) for _ in range(nf)]
        for h, f in zip(host_in, fs):
            h.copy_(torch.from_numpy(f))
        assert all(h.is_pinned() for h in host_in + host_out)
        plans = [fft3d.Plan(shape, torch.float32) for _ in range(nf)]
        dreal = [torch.empty(shape, dtype=torch.float32, device="cuda") for _ in range(nf)]
        cplx = [p.empty_complex() for p in plans]
        spectra = [torch.empty_like(c) for c in cplx]
        streams = [torch.cuda.Stream() for _ in range(nf)]
        torch.cuda.synchronize()
        for rnd in range(2):
            for i in range(nf):
                with torch.cuda.stream(streams[i]):
                    dreal[i].copy_(host_in[i], non_blocking=True)
                    plans[i].r2c(dreal[i], cplx[i])
                    spectra[i].copy_(cplx[i])
                    plans[i].c2r_overwrite(cplx[i], dreal[i])
                    host_out[i].copy_(dreal[i], non_blocking=True)
        torch.cuda.synchronize()
        ref_plan = fft3d.Plan(shape, torch.float32)
        for i in range(nf):
            X = ref_plan.r2c(torch.from_numpy(fs[i]).cuda())
            assert torch.equal(spectra[i], X)
            assert rel_l2(spectra[i].cpu().numpy(), F_refs[i]) <= TOL["f32"]
            y = ref_plan.c2r_overwrite(X.clone())
            torch.cuda.synchronize()
            assert torch.equal(host_out[i], y.cpu())
            assert rel_l2(host_out[i].numpy(), fs[i]) <= TOL["f32"]
    finally:
        hb.release()
