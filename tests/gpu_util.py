"""Shared helpers for the GPU tests: run the library on numpy inputs and
compare with the FP64 oracle."""
import numpy as np

TOL = {"f64": 1e-13, "f32": 5e-6}


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    n = np.linalg.norm(b.ravel())
    return np.linalg.norm((a - b).ravel()) / (n if n > 0 else 1.0)


def torch_dtype(name):
    import torch
    return torch.float32 if name == "f32" else torch.float64


def np_round(f, name):
    """The input as the library sees it: FP64 rounded once to FP32 for f32."""
    return f.astype(np.float32).astype(np.float64) if name == "f32" else f


def gpu_r2c(f, name, inplace=False):
    import torch
    import paper_2202_12756_gb300 as fft3d
    dt = torch_dtype(name)
    plan = fft3d.get_plan(f.shape, dt, "cuda")
    n2 = f.shape[2]
    if inplace:
        buf = plan.empty_padded()
        buf.fill_(float("nan"))
        buf[..., :n2].copy_(torch.from_numpy(f).to(dt))
        X = plan.r2c_(buf)
    else:
        x = torch.from_numpy(f).to(dt).cuda()
        X = plan.empty_complex()
        X.view(dt).fill_(float("nan"))
        plan.r2c(x, X)
    torch.cuda.synchronize()
    return X.cpu().numpy().astype(np.complex128)


def gpu_c2r(F, shape, name, inplace=False):
    import torch
    import paper_2202_12756_gb300 as fft3d
    dt = torch_dtype(name)
    plan = fft3d.get_plan(shape, dt, "cuda")
    cdt = fft3d.complex_of(dt)
    if inplace:
        buf = plan.empty_padded()
        buf.view(cdt).copy_(torch.from_numpy(F).to(cdt))
        out = plan.c2r_(buf)[..., : shape[2]]
    else:
        X = torch.from_numpy(F).to(cdt).cuda()
        out = plan.empty_real()
        out.fill_(float("nan"))
        plan.c2r(X, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)
