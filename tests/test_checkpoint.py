"""Checkpoints of provisioning results: applied only when device, parameters and revision match (host logic)."""
import json

from paper_2606_10477_gb300 import checkpoint, inputs


class FakeContext:
    def __init__(self, fwd=3, inv=5, modup=None, finish=None):
        self.v = {"forward": fwd, "inverse": inv, "modup": fwd if modup is None else modup,
                  "finish": fwd if finish is None else finish}

    def ntt_get_roles(self):
        return dict(self.v)

    def ntt_set_roles(self, roles):
        self.v.update(roles)


class FakeServer:
    table = None

    def set_table(self, R):
        self.table = R


R = [{"level": 12, "degree": 62, "c": 0, "iters": 7, "mre": 1.9e-9, "ms": 51.0, "kind": 1}]


def test_round_trip_applies_on_a_matching_key(tmp_path):
    p = inputs.PRESETS["bts16f"]
    path = str(tmp_path / "ckpt.json")
    checkpoint.save(path, FakeContext(2, 6, 1, 5), p, R, device="GPU A", git="abc")
    ctx, srv = FakeContext(0, 0), FakeServer()
    assert checkpoint.load(path, ctx, p, srv, device="GPU A", git="abc")
    assert ctx.v == {"forward": 2, "inverse": 6, "modup": 1, "finish": 5} and srv.table == R
    doc = json.load(open(path))
    assert doc["key"]["device"] == "GPU A" and doc["key"]["params"]["log_n"] == 16


def test_mismatched_key_or_missing_file_changes_nothing(tmp_path):
    p = inputs.PRESETS["bts16f"]
    path = str(tmp_path / "ckpt.json")
    checkpoint.save(path, FakeContext(2, 6), p, R, device="GPU A", git="abc")
    for kw, params in (({"device": "GPU B", "git": "abc"}, p), ({"device": "GPU A", "git": "def"}, p),
                       ({"device": "GPU A", "git": "abc"}, inputs.PRESETS["bts16"])):
        ctx, srv = FakeContext(0, 0), FakeServer()
        assert not checkpoint.load(path, ctx, params, srv, **kw)
        assert ctx.v == FakeContext(0, 0).v and srv.table is None
    assert not checkpoint.load(str(tmp_path / "none.json"), FakeContext(), p, device="GPU A", git="abc")
