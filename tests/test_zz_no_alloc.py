"""mor_solve_reduced_noalloc (the allocation-free reduced solve) against mor_solve_reduced.

Some callers cannot let a library allocate device memory: an application whose device
memory belongs to its own allocator or pool, or a time-critical loop that cannot take
cudaMalloc's implicit synchronization.  mor_solve_reduced_noalloc serves them with a
fixed device work array inside the library.  This test builds the reduced system of the
16^3 workload through the handle API, hands the same block-sparse matrix and load to the
allocation-free entry point through the C ABI (inputs and output allocated here by the
test), and checks two calls in a row against the handle solve within the 1e-10 relative
tolerance used for the reduced solution elsewhere.  The second call must leave the
device's free memory and PyTorch's allocated memory unchanged: after the first call on
a device has set up the fixed array, the entry point allocates nothing.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _block_sparse(K, n_sub, kq):
    """Neighbour lists and off-diagonal blocks of a dense reduced matrix (block row i:
    its nonzero blocks (i, j), j != i, in increasing j)."""
    ptr, sub, blk, blocks = [0], [], [], []
    for i in range(n_sub):
        for j in range(n_sub):
            if i == j:
                continue
            B = K[i * kq:(i + 1) * kq, j * kq:(j + 1) * kq]
            if np.any(B != 0.0):
                sub.append(j)
                blk.append(len(blocks))
                blocks.append(np.ascontiguousarray(B))
        ptr.append(len(sub))
    return (np.array(ptr, np.int32), np.array(sub, np.int32), np.array(blk, np.int32),
            np.stack(blocks).ravel())


def test_noalloc_reduced_solve_matches_handle_solve():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor

    mesh, kappa, owner, p = synth.workload("cube16_p2")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    opts = mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                          precision="fp64", cg_rtol=1e-13)
    bases = mor.Bases(sd, opts)
    red = mor.Reduced(sd, bases)
    x_ref, info_ref = red.solve(rtol=1e-13)
    x_ref = x_ref.cpu().numpy()
    assert info_ref["converged"]

    n_sub, kq = sd.n_sub, bases.kq
    ptr, sub, blk, blocks = _block_sparse(red.dense(), n_sub, kq)
    dev = "cuda"
    ptr_d = torch.as_tensor(ptr, device=dev)
    sub_d = torch.as_tensor(sub, device=dev)
    blk_d = torch.as_tensor(blk, device=dev)
    blocks_d = torch.as_tensor(blocks, device=dev)
    bt_d = torch.as_tensor(bases.bt().ravel(), device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    # both outputs are allocated before the first call, so that nothing else allocates
    # between the two calls
    xs = [torch.full((n_sub * kq,), float("nan"), dtype=torch.float64, device=dev)
          for _ in range(2)]
    torch.cuda.synchronize()
    mem = None
    for call in range(2):
        x_d = xs[call]
        info = mor.SolveInfo()
        rc = mor._lib.mor_solve_reduced_noalloc(n_sub, kq, P(ptr_d), P(sub_d), P(blk_d),
                                                P(blocks_d), P(bt_d), 1e-13, 20000, stream,
                                                P(x_d), ctypes.byref(info))
        assert rc == 0, mor._lib.mor_last_error()
        torch.cuda.synchronize()
        now = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated())
        if mem is not None:
            assert now == mem, "the second call changed device memory use: %s -> %s" % (mem, now)
        mem = now
        x = x_d.cpu().numpy()
        assert info.converged == 1
        assert np.max(np.abs(x - x_ref)) <= 1e-10 * np.max(np.abs(x_ref)), call
        assert abs(info.energy - info_ref["energy"]) <= 1e-10 * info_ref["energy"], call


def test_noalloc_rejects_systems_beyond_its_fixed_scratch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor
    one = torch.zeros(8, dtype=torch.float64, device="cuda")
    idx = torch.zeros(8, dtype=torch.int32, device="cuda")
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    # each limit on its own: too many subdomains (dim within its limit), and too many
    # unknowns (subdomains within theirs)
    for n_sub, kq in ((65537, 1), (1000, 600)):
        rc = mor._lib.mor_solve_reduced_noalloc(n_sub, kq, P(idx), P(idx), P(idx), P(one),
                                                P(one), 1e-10, 10, None, P(one), None)
        assert rc == -1, (n_sub, kq)
        assert b"too large" in mor._lib.mor_last_error()
