"""GPU parity of Algorithm 2 (Section 2.2), FGMRES(m_out)-GMRES_SP(m_in), on
the seeded stand-ins of the paper's Table 2 matrices, against the CPU oracle
(oracle/fgmres.py): the CSR product in FP64 and FP32 element by element, one
inner GMRES cycle (FP64: the same iterate; FP32: the same minimal residual
to FP32 accuracy), and whole solves (backward error recomputed here in FP64,
forward error against the oracle's solution within 10 kappa u64)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fgmres as fg
from paper_0808_2794_gb300 import inputs

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    return t


@pytest.fixture(scope="module")
def solver():
    from paper_0808_2794_gb300 import solver as s
    s.load()
    return s


def _dev(torch, ip, ix, d):
    return (torch.from_numpy(np.ascontiguousarray(ip)).cuda(), torch.from_numpy(np.ascontiguousarray(ix)).cuda(),
            torch.from_numpy(np.ascontiguousarray(d)).cuda())


def _system(name, n_target, seed):
    cfg = inputs.SPARSE_CONFIGS[name]
    scale = (n_target ** (1 / 3)) / cfg["g"] if cfg["kind"] == "stencil27" else n_target / cfg["n"]
    return inputs.sparse_system(name, scale=scale, seed=seed)


def _bwd(ip, ix, d, b, x):
    n = len(ip) - 1
    A = sp.csr_matrix((d, ix, ip), shape=(n, n))
    r = b - A @ x
    an = np.max(np.asarray(abs(A).sum(axis=1)).ravel())
    return np.max(np.abs(r)) / (an * np.max(np.abs(x)) + np.max(np.abs(b)))


@pytest.mark.parametrize("name", ["cage11_like", "poisson3db_like", "sio_like"])
def test_csr_spmv_fp64(torch, solver, name):
    """FP64 product: every row within 2 k u64 sum |a_ij x_j| of the oracle's
    (k = stored entries of the row; both sum in different orders)."""
    ip, ix, d, b, xt, _ = _system(name, 5000, seed=3)
    x = np.random.default_rng(1).standard_normal(len(ip) - 1)
    y = solver.csr_spmv(*_dev(torch, ip, ix, d), torch.from_numpy(x).cuda(), prec="fp64").cpu().numpy()
    want = fg.csr_matvec(ip, ix, d, x)
    k = np.diff(ip).astype(np.float64)
    bound = 2 * k * U64 * fg.csr_matvec(ip, ix, np.abs(d), np.abs(x))
    assert np.all(np.abs(y - want) <= bound + 1e-300)


@pytest.mark.parametrize("name", ["cage11_like", "sio_like"])
def test_csr_spmv_fp32(torch, solver, name):
    """FP32 product: values and x rounded to FP32 (RNE) and summed in FP32;
    every row within 2 k u32 sum |fl(a)| |fl(x)| of the oracle's FP32 product."""
    ip, ix, d, b, xt, _ = _system(name, 5000, seed=4)
    x = np.random.default_rng(2).standard_normal(len(ip) - 1)
    y = solver.csr_spmv(*_dev(torch, ip, ix, d), torch.from_numpy(x).cuda(), prec="fp32").cpu().numpy()
    d32, x32 = d.astype(np.float32), x.astype(np.float32)
    want = fg.csr_matvec(ip, ix, d32, x32).astype(np.float64)
    k = np.diff(ip).astype(np.float64)
    bound = 2 * k * U32 * fg.csr_matvec(ip, ix, np.abs(d32).astype(np.float64), np.abs(x32).astype(np.float64))
    assert np.all(np.abs(y - want) <= bound)
    # and it is the FP32 product, not the FP64 one
    y64 = fg.csr_matvec(ip, ix, d, x)
    assert np.max(np.abs(y - y64)) > 0


@pytest.mark.parametrize("m", [1, 5, 12])
def test_gmres_cycle_fp64_matches_oracle(torch, solver, m):
    """One FP64 inner cycle: the same number of steps and the same iterate as
    the oracle's textbook cycle (modified against classical Gram-Schmidt
    applied twice: agreement at rounding level for this well-conditioned A)."""
    ip, ix, d, b, xt, _ = _system("cage11_like", 3000, seed=5)
    v = b / np.linalg.norm(b)
    z, steps = solver.sparse_gmres_cycle(*_dev(torch, ip, ix, d), torch.from_numpy(v).cuda(), m, inner="fp64")
    ref = fg.gmres_cycle(ip, ix, d, v, m, np.float64)
    assert steps == ref["steps"]
    z = z.cpu().numpy()
    assert np.max(np.abs(z - ref["z"])) <= 1e-11 * np.max(np.abs(ref["z"]))


@pytest.mark.parametrize("name,m", [("cage11_like", 10), ("poisson3db_like", 20), ("sio_like", 30)])
def test_gmres_cycle_fp32_matches_oracle(torch, solver, name, m):
    """One FP32 inner cycle (GMRES_SP): GMRES minimises ||v - A z|| over the
    Krylov space, so the GPU's residual equals the oracle's to FP32 accuracy,
    and the two iterates agree to the FP32 level of this cycle."""
    ip, ix, d, b, xt, _ = _system(name, 4000, seed=6)
    v = b / np.linalg.norm(b)
    z, steps = solver.sparse_gmres_cycle(*_dev(torch, ip, ix, d), torch.from_numpy(v).cuda(), m, inner="fp32")
    z = z.cpu().numpy()
    ref = fg.gmres_cycle(ip, ix, d, v, m, np.float32)
    zr = ref["z"].astype(np.float64)
    n = len(ip) - 1
    A = sp.csr_matrix((d, ix, ip), shape=(n, n))
    res_gpu = np.linalg.norm(v - A @ z)
    res_or = np.linalg.norm(v - A @ zr)
    assert abs(steps - ref["steps"]) <= 1
    assert res_gpu <= 1.05 * res_or + 1e-5
    assert np.max(np.abs(z - zr)) <= 1e-4 * np.max(np.abs(zr))


@pytest.mark.parametrize("inner", ["fp32", "fp64", "none"])
@pytest.mark.parametrize("name", ["cage11_like", "poisson3db_like", "sio_like"])
def test_fgmres_parity(torch, solver, name, inner):
    """Whole solves at a few thousand unknowns: backward error <= 1e-14
    (recomputed here), forward error against the oracle's solution of the same
    method within 10 kappa_inf u64 (kappa from the dense inverse), and the
    outer-step count close to the oracle's."""
    ip, ix, d, b, xt, cfg = _system(name, 2000, seed=7)
    n = len(ip) - 1
    m_out, m_in = cfg["m_out"], cfg["m_in"]
    if inner == "none":
        m_out = cfg["m"]
    x, st = solver.fgmres(*_dev(torch, ip, ix, d), torch.from_numpy(b).cuda(), m_out=m_out, m_in=m_in,
                          inner=inner)
    x = x.cpu().numpy()
    assert st["flags"] == 0, st
    assert _bwd(ip, ix, d, b, x) <= 1e-14
    if inner == "none":
        ref = fg.gmres_restarted(ip, ix, d, b, m_out)
    else:
        ref = fg.fgmres(ip, ix, d, b, m_out, m_in, inner=np.float32 if inner == "fp32" else np.float64)
    assert ref["converged"]
    A = sp.csr_matrix((d, ix, ip), shape=(n, n)).toarray()
    kappa = np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf)
    fwd = np.max(np.abs(x - ref["x"])) / np.max(np.abs(ref["x"]))
    assert fwd <= 10 * kappa * U64, (fwd, kappa)
    steps_ref = ref["outer_steps"] if inner != "none" else ref["steps"]
    assert abs(st["outer_steps"] - steps_ref) <= max(2, steps_ref // 4), (st, steps_ref)
    if inner != "none":
        assert st["inner_steps"] > st["outer_steps"]


@pytest.mark.parametrize("name", ["cage11_like", "poisson3db_like", "sio_like"])
def test_fgmres_full_size(torch, solver, name):
    """The Table 2 stand-ins at their full orders (n = 39082, 85184, 33401):
    backward error <= 1e-14 recomputed here, and the solution agrees with the
    oracle's run of the same method and with x_true."""
    ip, ix, d, b, xt, cfg = inputs.sparse_system(name, seed=0)
    x, st = solver.fgmres(*_dev(torch, ip, ix, d), torch.from_numpy(b).cuda(), m_out=cfg["m_out"],
                          m_in=cfg["m_in"], inner="fp32")
    x = x.cpu().numpy()
    assert st["flags"] == 0, st
    assert _bwd(ip, ix, d, b, x) <= 1e-14
    ref = fg.fgmres(ip, ix, d, b, cfg["m_out"], cfg["m_in"], inner=np.float32)
    assert np.max(np.abs(x - ref["x"])) <= 1e-9 * np.max(np.abs(ref["x"]))
    assert np.max(np.abs(x - xt)) <= 1e-9


def test_fgmres_edge_cases(torch, solver):
    """n = 1; the identity (one outer step); b = 0 (x = 0 at once); m_in = 1."""
    one = _dev(torch, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([4.0]))
    x, st = solver.fgmres(*one, torch.tensor([2.0], dtype=torch.float64).cuda(), m_out=3, m_in=2)
    assert abs(float(x[0]) - 0.5) <= 1e-16 and st["flags"] == 0
    n = 1000
    eye = _dev(torch, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    b = np.random.default_rng(0).standard_normal(n)
    # an FP64 inner cycle returns z = v exactly: one outer step; the FP32 one
    # returns fl32(v), so the outer method needs a second step
    x, st = solver.fgmres(*eye, torch.from_numpy(b).cuda(), m_out=5, m_in=5, inner="fp64")
    assert np.max(np.abs(x.cpu().numpy() - b)) <= 1e-15 * np.max(np.abs(b)) and st["outer_steps"] == 1
    x, st = solver.fgmres(*eye, torch.from_numpy(b).cuda(), m_out=5, m_in=5)
    # (accurate to the backward-error target: for A = I the error is the residual)
    assert np.max(np.abs(x.cpu().numpy() - b)) <= 2e-14 * np.max(np.abs(b)) and st["outer_steps"] <= 3
    x, st = solver.fgmres(*eye, torch.zeros(n, dtype=torch.float64).cuda())
    assert float(x.abs().max()) == 0.0 and st["cycles"] == 0 and st["flags"] == 0
    ip, ix, d, b, xt, _ = _system("cage11_like", 1500, seed=8)
    x, st = solver.fgmres(*_dev(torch, ip, ix, d), torch.from_numpy(b).cuda(), m_out=10, m_in=1)
    assert st["flags"] == 0 and _bwd(ip, ix, d, b, x.cpu().numpy()) <= 1e-14


def test_fgmres_argument_errors(torch, solver):
    import ctypes
    lib = solver.load()
    o = solver.sparse_opts()
    o.m_out = 0
    assert lib.mp_fgmres(10, 10, None, None, None, None, None, None, 0, ctypes.byref(o), None, None) == -3
    assert lib.mp_fgmres(-1, 0, None, None, None, None, None, None, 0, ctypes.byref(o), None, None) == -1
    ip, ix, d = _dev(torch, np.arange(11, dtype=np.int32), np.arange(10, dtype=np.int32), np.ones(10))
    b = torch.ones(10, dtype=torch.float64).cuda()
    x = torch.empty(10, dtype=torch.float64).cuda()
    assert lib.mp_fgmres(10, 10, ip.data_ptr(), ix.data_ptr(), d.data_ptr(), b.data_ptr(), x.data_ptr(), None, 0,
                         ctypes.byref(o), None, None) == -10
    o = solver.sparse_opts()
    assert lib.mp_fgmres(10, 10, ip.data_ptr(), ix.data_ptr(), d.data_ptr(), b.data_ptr(), x.data_ptr(), None, 0,
                         ctypes.byref(o), None, None) == -9
