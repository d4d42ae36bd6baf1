"""The library's device pool: freed blocks stay cached for later
allocations, ed_memory_trim returns them, and results do not depend on
whether the memory a solve gets was cached or fresh."""
import pytest

from workloads import workload_ns14

pytestmark = pytest.mark.gpu


def test_pool_caches_reuses_and_trims(ed):
    wl = workload_ns14(0)                      # D = 11,778,624
    s = ed.Sector(wl.model, wl.nup, wl.ndw)
    vec = s.blocked_dim * 4                    # one FP32 block-major vector
    r1 = ed.lanczos_ground(s, "fp32_polish")
    reserved, used = ed.memory_cached()
    # the solve's workspace (at least three FP32 vectors) was freed into the
    # pool and is still reserved there; only the sector's tables are in use
    assert reserved - used >= 3 * vec
    r2 = ed.lanczos_ground(s, "fp32_polish")   # on the cached blocks
    reserved2, _ = ed.memory_cached()
    assert reserved2 <= reserved + vec         # reused, not grown by another solve's worth
    ed.trim_memory()
    reserved3, used3 = ed.memory_cached()
    assert reserved3 < reserved2 and used3 <= reserved3
    r3 = ed.lanczos_ground(s, "fp32_polish")   # on fresh memory again
    for r in (r2, r3):
        assert r["e0"] == r1["e0"] and r["iterations"] == r1["iterations"]
    with pytest.raises(ed.EDError):
        ed.trim_memory(-1)
    s.free()
