"""Host-side figures of bench.py's roofline: the FLOP attribution per phase and the DRAM traffic record.

* In the tiled layout (Euler, orders 2-3) the predictor kernel solves every face once, so its FLOPs per
  zone are the predictor's and faces' plus the face solves' (the HLL update's count less Eq. 6's own
  FLOPs), and the update phase carries only Eq. 6; the per-zone layout keeps the counter's phases.
* The traffic record scales to a launch in proportion to the zones, and only for the configuration and
  the source files it was captured with (a changed source gives None).
"""
import importlib.util
import json
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(root=ROOT):
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _flops():
    with open(os.path.join(ROOT, "paper_1006_2146_gb300", "flops.json")) as fh:
        return json.load(fh)


def test_tiled_flop_attribution():
    b = _bench()
    f = _flops()["order3"]
    t = b.flops_per_zone(3, "nodal", "hll", False, tiled=True)
    assert t["riemann_update"] == b.UPDATE_FLOPS
    assert t["predictor_faces"] == f["predictor_faces_nodal"] + f["riemann_update_hll"] - b.UPDATE_FLOPS
    assert t["weno_reconstruction"] == f["weno_reconstruction"]
    # the whole step's count is the same in either attribution
    z = b.flops_per_zone(3, "nodal", "hll", False, tiled=False)
    assert sum(t.values()) == sum(z.values())
    # order 4 has no tiled layout: the counter's phases
    o4 = b.flops_per_zone(4, "modal", "hll", True, tiled=True)
    assert o4["riemann_update"] == _flops()["order4"]["riemann_update_fused_hll"]


def test_traffic_record_scales_and_checks_its_sources(tmp_path):
    b = _bench()
    with open(os.path.join(ROOT, "profiles", "traffic_predictor_faces.json")) as fh:
        rec = json.load(fh)
    zones = 256 ** 3
    got = b.traffic_per_launch("predictor_faces", rec["order"], rec["form"], rec["precision"] == "fp32", zones)
    assert got == rec["bytes_per_zone"] * zones
    assert b.traffic_per_launch("predictor_faces", 4, rec["form"], False, zones) is None
    # a copy of the tree with one listed source changed: the record no longer applies
    shutil.copy(os.path.join(ROOT, "bench.py"), tmp_path / "bench.py")
    for rel in rec["sources"] + ["profiles/traffic_predictor_faces.json"]:
        dst = tmp_path / rel
        os.makedirs(dst.parent, exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), dst)
    b2 = _bench(str(tmp_path))
    assert b2.traffic_per_launch("predictor_faces", rec["order"], rec["form"], False, zones) == got
    with open(tmp_path / rec["sources"][0], "a") as fh:
        fh.write("\n// changed\n")
    assert b2.traffic_per_launch("predictor_faces", rec["order"], rec["form"], False, zones) is None
