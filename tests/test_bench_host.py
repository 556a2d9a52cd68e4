"""Host-side reporting in bench.py (no GPU): the rounds of a fused gate call
from its public shape, and the network projection T_comp + 2 B / BW + R RTT
(the paper's Eq. for projected online latency, LAN 1 GB/s / 0.5 ms and WAN
400 MB/s / 4 ms) on the BERT-base layer's byte and round counts."""
import numpy as np
import pytest

import bench
from paper_2606_09551_b300 import fusefss as F
from paper_2606_09551_b300 import inputs as I
from paper_2606_09551_b300 import specs as S


def _shape(sp):
    return F.CompiledSpec(sp).shape      # host-only compile


def test_op_rounds_from_shape():
    assert bench.op_rounds(_shape(S.gelu8())) == 1 + 2          # opening + two Horner rounds
    assert bench.op_rounds(_shape(S.nexp16())) == 1 + 3
    assert bench.op_rounds(_shape(S.gelu8().variant(True))) == 1  # x^ basis: local Horner
    assert bench.op_rounds(_shape(S.trunc(32, 12, True))) == 2    # opening + the daBit byte
    pw = S.random_piecewise(np.random.default_rng(3), S.gelu4(), 2)
    sh = _shape(pw)
    assert bench.op_rounds(sh) == 1 + 2 + sh.bx_rounds


def test_network_projection_bert_layer():
    calls = I.bert_layer()
    css = {c.name: F.CompiledSpec(c.spec) for c in calls}
    b = sum(c.n * (8 + 16 * c.spec.degree) for c in calls)      # 8 + 16 d bytes per element
    p = bench.network_projection(calls, css, 10.0, [b * 3, b * 3], 3)
    assert p["comm_bytes_per_party"] == b and p["counted_bytes_match"]
    assert p["rounds"] == 3 + 4 + 4 + 4
    assert p["lan"]["t_proj_ms"] == pytest.approx(10.0 + 2e3 * b / 1e9 + 15 * 0.5)
    assert p["wan"]["t_proj_ms"] == pytest.approx(10.0 + 2e3 * b / 400e6 + 15 * 4.0)
    assert not bench.network_projection(calls, css, 10.0, [b * 3 + 1, b * 3], 3)["counted_bytes_match"]


def test_tuning_replay_installs_saved_records(tmp_path):
    """--tuning-from: the last JSON line's autotune records give each call
    its saved arity and layout, and the saved model is installed (host-only
    compile, so the arity and layout are checked on the compiled shape)."""
    import json
    rec = {"slots": [1, 2, 4], "tile_us": [200.0, 100.0, 60.0], "fixed_us": [2.0, 1.0, 1.0],
           "sample_elems": 75776, "dealer_ms": 10.0, "dcf_bits": 6, "lookup_records": True,
           "dcf_bits_chosen_by": "measured, form 0 at 393216 elements"}
    path = tmp_path / "run.json"
    path.write_text("log line\n" + json.dumps({"autotune": {"gelu": dict(rec, dcf_bits=3)}}) + "\n"
                    + json.dumps({"autotune": {"gelu": rec}}) + "\n")
    saved = bench.load_tuning(str(path))
    assert saved["gelu"]["dcf_bits"] == 6

    class Args:
        dcf_bits, no_autotune, records = 0, False, False
    calls = [c for c in I.bert_layer() if c.name == "gelu"]
    css = bench.compile_specs(None, calls, Args(), form=0, replay=saved)
    cs = css["gelu"]
    assert cs.spec.dcf_bits == 6 and cs.records and cs.shape.dcf_bits == 6 and cs.shape.lookup_records == 1
    assert cs.arity_choice.startswith("replayed")
