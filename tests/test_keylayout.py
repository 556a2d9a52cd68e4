"""The test-side restatement of the library's key layout (tests/keylayout.py)
is consistent with itself and with the library (CPU only): oracle key
records packed into the layout read back field for field, and the layout's
total size equals what the library allocates for the same spec and n."""
import numpy as np
import pytest

import oracle as O
from keylayout import fields_equal, gpu_fields, offsets, oracle_fields, oracle_to_gpu
from paper_2606_09551_b300 import fusefss as F
from paper_2606_09551_b300 import inputs as I
from paper_2606_09551_b300 import specs as S

SPECS = [S.gelu4(), S.gelu8(), S.nexp16(), S.trunc(32, 12, True), S.relu(5),
         S.random_spec(np.random.default_rng(4), 12, 5, 1, 2, n_extra=2, name="rand_r2")]


@pytest.mark.parametrize("records", [False, True])
@pytest.mark.parametrize("dcf_bits", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("sp", SPECS, ids=[s.name for s in SPECS])
def test_layout_round_trip_and_size(sp, dcf_bits, records):
    sp = sp.arity(dcf_bits)
    osp = O.Spec(**sp.descriptor())
    n = 37
    x = I.uniform_x(n, sp.k, 3)
    k0, _, _, _ = O.dealer(osp, I.KEY_SEED, 9, 0, n, x)
    buf = oracle_to_gpu(k0, osp, n, records)
    if records and osp.M > 1 and osp.p not in (3, 4):
        with pytest.raises(F.FfssError):        # records are built for p = 3, 4 lookups
            F.CompiledSpec(sp, records=True)
        return
    cs = F.CompiledSpec(sp, records=records)
    assert cs.records == (records and osp.M > 1)
    assert buf.size == offsets(osp, n, records)["total"] == cs.key_bytes(n)
    for e in (0, 1, n - 1):
        assert fields_equal(gpu_fields(buf, osp, n, e, records), oracle_fields(k0, osp, e)), e
