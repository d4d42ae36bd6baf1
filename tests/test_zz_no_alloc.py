"""ed_residual_noalloc: the allocation-free residual check, for callers that
cannot let a library allocate device memory (applications that give all
device memory to their own pool allocator, latency-critical loops in which
cudaMalloc/cudaFree could block).

It is compared with the entry points that allocate: the Lanczos ground state
(its energy and FP64 residual) and ed_matvec (the product it re-computes),
on two calls in a row, in the FP64 tolerance of the other GPU tests.  This
file is collected last so that a failure here does not stop the rest."""
import numpy as np
import pytest
import torch

from workloads import make_model, with_exchange, workload_ns8

def _reference(ed, s, psi):
    """E and ||H psi - E psi|| / ||psi|| through ed_matvec (allocating path)."""
    w = torch.empty_like(psi)
    ed.matvec(s, psi, w, "fp64")
    nn = float(torch.dot(psi, psi))
    e = float(torch.dot(psi, w)) / nn
    r = float(torch.linalg.norm(w - e * psi)) / nn ** 0.5
    return e, r


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["ns8", "norb2_ns10", "kanamori_norb3_ns9"])
def test_noalloc_matches_allocating_entry_points(ed, case):
    if case == "ns8":
        m, nup, ndw = workload_ns8().model, 4, 4
    elif case == "norb2_ns10":
        m, nup, ndw = make_model(2, 4, U=3.0, Jh=0.5, seed=6), 5, 5
    else:   # spin exchange and pair hopping
        m, nup, ndw = with_exchange(make_model(3, 2, U=2.6, Jh=0.4, seed=31), 0.35, 0.3), 4, 5
    s = ed.Sector(m, nup, ndw)
    assert s.dim <= 1 << 20
    psi = torch.empty(s.dim, dtype=torch.float64, device="cuda")
    res = ed.lanczos_ground(s, "fp64", psi=psi)
    first = ed.residual_noalloc(s, psi)
    second = ed.residual_noalloc(s, psi)
    assert first == second                       # two calls in a row, same scratch
    e, r = first
    assert abs(e - res["e0"]) <= 1e-10 * abs(res["e0"])
    assert abs(r - res["residual"]) <= 1e-12
    e_ref, r_ref = _reference(ed, s, psi)
    assert abs(e - e_ref) <= 1e-12 * abs(e_ref)
    assert abs(r - r_ref) <= 1e-12
    # a vector far from an eigenvector: residual of order one
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.rand(s.dim, dtype=torch.float64, device="cuda", generator=g) - 0.5
    a1 = ed.residual_noalloc(s, x)
    a2 = ed.residual_noalloc(s, x)
    assert a1 == a2
    e_ref, r_ref = _reference(ed, s, x)
    assert abs(a1[0] - e_ref) <= 1e-12 * max(1.0, abs(e_ref))
    assert abs(a1[1] - r_ref) <= 1e-12 * max(1.0, r_ref)
    s.free()


@pytest.mark.gpu
def test_noalloc_rejects_oversized_and_mismatched(ed):
    from workloads import workload_ns14
    wl = workload_ns14(0)
    s = ed.Sector(wl.model, 7, 7)            # D = 11,778,624 > 2**20
    x = torch.zeros(s.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(ed.EDError) as e:
        ed.residual_noalloc(s, x)
    assert e.value.status == ed.ED_ERR_ARG
    s.free()
    s = ed.Sector(workload_ns8().model, 4, 4)
    with pytest.raises(ed.EDError) as e:
        ed.residual_noalloc(s, torch.zeros(s.dim + 1, dtype=torch.float64, device="cuda"))
    assert e.value.status == ed.ED_ERR_ARG
    s.free()
    # a float32 vector (as the FP32 ground state returns) is refused before
    # the library reads it as doubles
    s = ed.Sector(workload_ns8().model, 4, 4)
    with pytest.raises(ed.EDError) as e:
        ed.residual_noalloc(s, torch.zeros(s.dim, dtype=torch.float32, device="cuda"))
    assert e.value.status == ed.ED_ERR_ARG
    s.free()


@pytest.mark.gpu
def test_noalloc_allocates_no_device_memory(ed):
    """After the first call on the device (which loads the module holding the
    static scratch array), further calls leave the free device memory as it
    was: nothing is allocated or released."""
    s = ed.Sector(make_model(2, 4, U=3.0, Jh=0.5, seed=6), 5, 5)
    g = torch.Generator(device="cuda").manual_seed(2)
    x = torch.rand(s.dim, dtype=torch.float64, device="cuda", generator=g) - 0.5
    first = ed.residual_noalloc(s, x)            # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert ed.residual_noalloc(s, x) == first
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    s.free()


def test_noalloc_binding_rejects_non_double_vectors():
    """CPU check of the binding's argument guard: a vector that is not a
    contiguous float64 CUDA tensor on the sector's device never reaches the
    C entry point (which would read it as doubles)."""
    import paper_2105_06806_gb300 as E

    class _FakeSector:
        h = None
        device = 0

    for bad in (torch.zeros(16, dtype=torch.float32), torch.zeros(16, dtype=torch.float64),
                torch.zeros(32, dtype=torch.float64)[::2]):
        with pytest.raises(E.EDError) as e:
            E.residual_noalloc(_FakeSector(), bad)
        assert e.value.status == E.ED_ERR_ARG
