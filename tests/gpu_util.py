"""Helpers shared by the GPU tests: run the CUDA path through the C ABI on seeded inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def make_ctx(el, s_prec="fp64", k_prec="fp64", symm=True, **kw):
    from paper_2203_15461_gb300.cpm import CPM
    return CPM.for_electrodes(el, s_prec=s_prec, k_prec=k_prec, symm=symm, **kw)


def stack_replicas(elyts, n_e=None):
    """Pack electrolytes replica-major, padding the shorter ones with Q = 0 charges."""
    n_e = n_e or max(e.n for e in elyts)
    xyz = np.zeros((len(elyts), n_e, 3))
    Q = np.zeros((len(elyts), n_e))
    for r, e in enumerate(elyts):
        xyz[r, :e.n] = e.xyz
        Q[r, :e.n] = e.Q
        xyz[r, e.n:] = e.xyz[0] if e.n else 0.0   # padding sits on a real charge's position; Q = 0 skips it
    return xyz.reshape(-1, 3), Q.reshape(-1), n_e


def run_bvec(ctx, elyts):
    xyz, Q, n_e = stack_replicas(elyts)
    m = len(elyts)
    b = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
    ctx.cpm_bvec(m, n_e, dev(xyz), dev(Q), b)
    torch.cuda.synchronize()
    return b.cpu().numpy()


def run_update(ctx, psi, b):
    m = b.shape[0]
    q = torch.empty((m, ctx.n), dtype=torch.float64, device="cuda")
    qt = torch.empty((m,), dtype=torch.float64, device="cuda")
    ctx.cpm_update(m, dev(np.tile(psi, (m, 1))), dev(b), q, qt)
    torch.cuda.synchronize()
    return q.cpu().numpy(), qt.cpu().numpy()
