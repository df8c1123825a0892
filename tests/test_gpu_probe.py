"""ac_probe_gather: the lookup ceilings the rooflines use.

A table in shared memory answers random lookups faster than one read
through L2, which is faster than one in HBM; bad arguments are refused.
"""
import pytest

from paper_1403_1305_gb300 import ac as A

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_ceilings_are_ordered():
    sm = A.ac_probe_gather(0, 64 << 10, shared=True, threads=1024, chains=4, steps=512)
    l2 = A.ac_probe_gather(0, 4 << 20, shared=False, threads=1024, chains=4, steps=512)
    hbm = A.ac_probe_gather(0, 1 << 30, shared=False, threads=1024, chains=4, steps=256)
    props = torch.cuda.get_device_properties(0)
    for r in (sm, l2, hbm):
        assert r["ms"] > 0 and r["sms"] == props.multi_processor_count and r["chains_per_sm"] == 4096
        assert r["gathers"] == r["sms"] * 4096 * (512 if r is not hbm else 256)
    assert sm["gathers_per_s"] > l2["gathers_per_s"] > hbm["gathers_per_s"]


def test_refusals():
    for kw, code in ((dict(threads=33), A.AC_EINVAL), (dict(chains=3), A.AC_EINVAL),
                     (dict(table_bytes=64), A.AC_ERANGE), (dict(table_bytes=1 << 20, shared=True), A.AC_ERANGE)):
        args = dict(table_bytes=1 << 20, shared=False, threads=256, chains=1, steps=16)
        args.update(kw)
        with pytest.raises(A.AcError) as e:
            A.ac_probe_gather(0, **args)
        assert e.value.code == code, kw


def test_launch_probe_in_a_graph():
    """ac_probe_launch enqueues empty kernels that a CUDA graph captures,
    one node each; replaying the graph runs them."""
    s = torch.cuda.Stream()
    A.ac_probe_launch(s, 3, 128, 512)  # outside a capture first
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        A.ac_probe_launch(torch.cuda.current_stream(), 6, 1, 32)
    g.replay()
    torch.cuda.synchronize()
