"""Multi-right-hand-side D_eo and the batched CG (through the C ABI).

* each field of a multi-RHS application equals the single-field FP32
  application bit for bit (same operations in the same order), for every
  batch size 1..16 and both link storages;
* against the FP64 oracle within the FP32 rounding bound;
* the batched CG reaches the FP64 true residual tol for every field,
  recomputed by the oracle, and equals independent solves within the
  conditioning bound."""
import numpy as np
import pytest
import torch

from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu


def batch_to_device(fields, dtype=torch.complex64):
    """[n][Vh][3] host -> device [3][Vh][n]."""
    a = np.ascontiguousarray(np.transpose(np.asarray(fields), (2, 1, 0)))
    return torch.from_numpy(a).to(dtype).cuda().contiguous()


def batch_from_device(t):
    return np.ascontiguousarray(np.transpose(t.cpu().numpy(), (2, 1, 0))).astype(np.complex128)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 12, 16])
@pytest.mark.parametrize("recon", [18, 12])
def test_mrhs_equals_single_rhs_bitwise(gpu, n, recon):
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims)
    fields = [inputs.gaussian_field(dims, k=j) for j in range(n)]
    with gpu.Context(dims) as c:
        c.links_upload(U)
        for parity in (0, 1):
            xin = batch_to_device(fields)
            out = torch.empty_like(xin)
            c.deo_apply_mrhs(parity, n, recon, xin, out)
            torch.cuda.synchronize()
            got = batch_from_device(out)
            for j in range(n):
                xs = gpu.to_device_spinor(fields[j], dtype=torch.complex64)
                os_ = torch.empty_like(xs)
                c.deo_apply_ex(parity, gpu.PREC_FP32, recon, xs, os_)
                torch.cuda.synchronize()
                assert np.array_equal(got[j], gpu.from_device_spinor(os_)), f"field {j}"


@pytest.mark.parametrize("n", [1, 3, 4, 16])
@pytest.mark.parametrize("recon", [18, 12])
def test_field_major_equals_site_major_bitwise(gpu, n, recon):
    """The field-major layout [3][n][Vh] gives, field by field, the bits of
    the site-major layout (and so of the single-field operator)."""
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims)
    fields = [inputs.gaussian_field(dims, k=j) for j in range(n)]
    with gpu.Context(dims) as c:
        c.links_upload(U)
        for parity in (0, 1):
            xs = batch_to_device(fields)                       # [3][Vh][n]
            os_ = torch.empty_like(xs)
            c.deo_apply_mrhs(parity, n, recon, xs, os_)
            xf = xs.permute(0, 2, 1).contiguous()              # [3][n][Vh]
            of = torch.empty_like(xf)
            c.deo_apply_mrhs(parity, n, recon, xf, of, layout=1)
            torch.cuda.synchronize()
            assert torch.equal(of.permute(0, 2, 1), os_)
        with pytest.raises(gpu.LqcdError):
            c.deo_apply_mrhs(0, n, recon, xf, of, layout=2)


@pytest.mark.parametrize("R", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("layout", [0, 1])
def test_every_fields_per_thread_variant_bitwise(gpu, monkeypatch, R, layout):
    """Each fields-per-thread choice of the tuner, forced, gives every field
    the bits of the single-field operator (n = 16, both layouts, 12-real and
    18-real links)."""
    n = 16
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims)
    fields = [inputs.gaussian_field(dims, k=j) for j in range(n)]
    monkeypatch.setenv("LQCD_MRHS_R", str(R))
    with gpu.Context(dims) as c:
        c.links_upload(U)
        for recon in (12, 18):
            xs = batch_to_device(fields)                       # [3][Vh][n]
            xin = xs if layout == 0 else xs.permute(0, 2, 1).contiguous()
            out = torch.empty_like(xin)
            c.deo_apply_mrhs(1, n, recon, xin, out, layout=layout)
            torch.cuda.synchronize()
            got = batch_from_device(out if layout == 0 else out.permute(0, 2, 1))
            for j in range(n):
                xsj = gpu.to_device_spinor(fields[j], dtype=torch.complex64)
                osj = torch.empty_like(xsj)
                c.deo_apply_ex(1, gpu.PREC_FP32, recon, xsj, osj)
                torch.cuda.synchronize()
                assert np.array_equal(got[j], gpu.from_device_spinor(osj)), f"R {R} field {j}"


@pytest.mark.parametrize("n", [4, 16])
def test_mrhs_unaligned_buffers_equal_aligned(gpu, n):
    """in / out 8 bytes off a 16-byte boundary take the one-field-per-access
    kernel and give the same bits as aligned buffers (two fields per access)."""
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims)
    fields = [inputs.gaussian_field(dims, k=j) for j in range(n)]
    with gpu.Context(dims) as c:
        c.links_upload(U)
        xin = batch_to_device(fields)
        out = torch.empty_like(xin)
        c.deo_apply_mrhs(0, n, 12, xin, out)
        m = xin.numel()
        bi = torch.empty(m + 1, dtype=torch.complex64, device="cuda")
        bo = torch.empty(m + 1, dtype=torch.complex64, device="cuda")
        xu, ou = bi[1:].view(xin.shape), bo[1:].view(xin.shape)
        xu.copy_(xin)
        assert xu.data_ptr() % 16 == 8 and ou.data_ptr() % 16 == 8
        c.deo_apply_mrhs(0, n, 12, xu, ou)
        torch.cuda.synchronize()
        assert torch.equal(ou, out)


def test_mrhs_against_oracle(gpu, orc):
    dims = (8, 8, 8, 8)
    n = 16
    U = inputs.random_links(dims)
    fields = [inputs.gaussian_field(dims, k=j) for j in range(n)]
    with gpu.Context(dims) as c:
        c.links_upload(U)
        xin = batch_to_device(fields)
        out = torch.empty_like(xin)
        c.deo_apply_mrhs(0, n, 12, xin, out)
        torch.cuda.synchronize()
        got = batch_from_device(out)
    for j in range(n):
        ref = orc.deo(dims, 0, U, fields[j])
        assert np.linalg.norm(got[j] - ref) / np.linalg.norm(ref) < 5e-6


@pytest.mark.parametrize("n", [1, 4, 5, 16])
def test_batched_cg(gpu, orc, n):
    dims = (8, 8, 8, 8)
    U = inputs.random_links(dims)
    b = np.stack([inputs.gaussian_field(dims, k=j) for j in range(n)])
    with gpu.Context(dims, prec=gpu.PREC_FP32, recon=12) as c:
        c.links_upload(U)
        x, infos = c.cg_solve_mrhs(0.1, 0.0, 1e-10, b)
    for j in range(n):
        r = orc.true_residual(dims, U, 0.1, 0.0, b[j], x[j])
        assert r <= 1e-10, f"field {j}: {r:.2e}"
        assert infos[j]["true_resid"][0] <= 1e-10
    xr, _ = orc.cg(dims, U, 0.1, 0.0, b[0], 1e-11)
    assert np.linalg.norm(x[0] - xr) / np.linalg.norm(xr) < 2 * (0.01 + 16) / 0.01 * 1e-10


def test_batched_cg_alone_equals_in_batch(gpu):
    """Field 0 of a batch of 8 gives the same solution as solved in a batch
    of 1 up to the rounding of the shared reliable-update schedule."""
    dims = (8, 8, 8, 8)
    U = inputs.random_links(dims)
    b = np.stack([inputs.gaussian_field(dims, k=j) for j in range(8)])
    with gpu.Context(dims, prec=gpu.PREC_FP32, recon=12) as c:
        c.links_upload(U)
        x8, _ = c.cg_solve_mrhs(0.1, 0.0, 1e-10, b)
        x1, _ = c.cg_solve_mrhs(0.1, 0.0, 1e-10, b[:1])
    assert np.linalg.norm(x8[0] - x1[0]) / np.linalg.norm(x1[0]) < 1e-7


def test_mrhs_argument_errors(gpu):
    dims = (4, 4, 4, 4)
    with gpu.Context(dims) as c:
        c.links_upload(inputs.random_links(dims))
        x = torch.zeros((3, c.Vh, 17), dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        with pytest.raises(gpu.LqcdError):
            c.deo_apply_mrhs(0, 17, 12, x, y)
        with pytest.raises(gpu.LqcdError):
            c.deo_apply_mrhs(0, 4, 10, x, y)
        with pytest.raises(gpu.LqcdError):
            c.cg_solve_mrhs(0.0, 0.0, 1e-10, np.ones((2, c.Vh, 3)))
