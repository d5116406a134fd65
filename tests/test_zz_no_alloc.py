"""The allocation-free trace entry point (isdf_eri_traces_noalloc).

Some callers cannot let a library allocate device memory: an application whose
own allocator owns the GPU's memory, or a latency-critical loop that cannot
take the implicit synchronisation of cudaMalloc.  For them the library offers
a handle-free trace reduction whose scratch is a fixed device array.  This
test checks, through the C ABI, that it reproduces the E_J / E_K that
isdf_fragment_eri returns, on two consecutive calls (the array keeps the
previous call's contents), and that sizes beyond its limit are refused.
"""
import numpy as np
import pytest

from paper_2601_16379_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-8   # the FP64 parity tolerance of the other GPU tests


def test_noalloc_traces_match_fragment_eri(cuda, lib_built):
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    wl = W.workload("c1")
    g = B.Isdf(wl.cell, B.ISDF_FP64)
    g.build_points(wl.n_p, wl.seed)
    g.fit_zeta(1e-7)
    g.coulomb_metric()
    frags = [wl.fragments[0], W.make_fragment(wl.cell, wl.seed, 7, 9)]
    Cs = [torch.from_numpy(f.C).cuda() for f in frags]
    gs = [torch.from_numpy(f.gamma).cuda() for f in frags]
    eris = [torch.empty((f.norb,) * 4, dtype=torch.complex128, device="cuda") for f in frags]
    ej, ek = g.fragment_eri(Cs, gs, eris)
    torch.cuda.synchronize()
    for call in range(2):
        for i, f in enumerate(frags):
            ej2, ek2 = B.eri_traces_noalloc(eris[i], f.norb, gs[i])
            assert abs(ej2 - ej[i]) < TOL, (call, i, ej2, ej[i])
            assert abs(ek2 - ek[i]) < TOL, (call, i, ek2, ek[i])
    g.close()


def test_noalloc_rejects_sizes_beyond_limit(cuda, lib_built):
    from paper_2601_16379_gb300 import binding as B
    torch = cuda
    small = torch.zeros(4, dtype=torch.complex128, device="cuda")
    with pytest.raises(B.IsdfError) as e:
        B.eri_traces_noalloc(small, 512, small)
    assert e.value.code == -1
    assert "511" in str(e.value)
