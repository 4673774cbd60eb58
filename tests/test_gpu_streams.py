"""Two streams transforming the same shape at the same time.

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
