"""The host-buffer gate (ffss_eval_pair_host): the end-to-end form copies
page-locked host input shares in, runs the fused gate and copies the output
shares out, all queued on the caller's stream.  Its shares equal the
device-buffer call's for the same keys; calls alternating between two
streams (sharing the context's two staging slots) stay correct, and a call
larger than the staging grows it."""
import numpy as np
import pytest

from paper_2606_09551_b300 import fusefss as F
from paper_2606_09551_b300 import inputs as I
from paper_2606_09551_b300 import specs as S

pytestmark = pytest.mark.gpu


def test_host_buffers_match_device_buffers():
    import torch
    from paper_2606_09551_b300 import build
    build.build()
    ctx = F.Context(0)
    specs = [S.gelu8(), S.nexp16(), S.relu(16)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for rep, n in enumerate((1000, 70000, 3000, 200000)):
        sp = specs[rep % len(specs)]
        cs = F.CompiledSpec(sp, ctx)
        x = torch.from_numpy(I.uniform_x(n, sp.k, 80 + rep)).cuda()
        sets = []
        for _ in range(2):
            k0, k1 = F.Keys(cs, n, 0), F.Keys(cs, n, 1)
            x0, x1 = torch.empty_like(x), torch.empty_like(x)
            F.keygen(ctx, cs, I.KEY_SEED, 500 + rep, n, k0, k1, x, x0, x1)
            sets.append((k0, k1, x0, x1))
        k0, k1, x0, x1 = sets[0]
        dev = [torch.empty(n * sp.n_out, dtype=torch.uint64, device="cuda:0") for _ in range(2)]
        dev += [torch.empty(n, dtype=torch.uint32, device="cuda:0") for _ in range(2)]
        F.eval_pair(ctx, cs, k0, k1, x0, x1, *dev)
        torch.cuda.synchronize()
        k0, k1, x0, x1 = sets[1]
        hx0, hx1 = x0.cpu().pin_memory(), x1.cpu().pin_memory()
        host = [torch.empty(n * sp.n_out, dtype=torch.uint64).pin_memory() for _ in range(2)]
        host += [torch.empty(n, dtype=torch.uint32).pin_memory() for _ in range(2)]
        st = streams[rep % 2]
        st.wait_stream(torch.cuda.current_stream())
        comm = torch.zeros(2, dtype=torch.uint64, device="cuda:0")
        F.eval_pair_host(ctx, cs, k0, k1, hx0, hx1, *host, comm=comm, stream=st)
        st.synchronize()
        for h, d in zip(host, dev):
            assert torch.equal(h, d.cpu()), (rep, sp.name)
        mults = sp.degree * sp.n_out
        assert comm.cpu().tolist() == [n * (8 + 16 * mults)] * 2
