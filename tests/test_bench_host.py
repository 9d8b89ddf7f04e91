"""Host logic of bench.py that needs no GPU: the source hash that decides whether the
committed ncu DRAM counters still describe the kernel being timed."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_host_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_comment_edits_keep_the_code_text_and_code_edits_change_it():
    b = _bench()
    src = "int f(int x)   // scale\n{\n    // twice\n    return 2 * x;\n}\n"
    commented = "// new header line\nint f(int x)   // scale by two\n{\n\n    return 2 * x;   // doubled\n}\n"
    changed = "int f(int x)   // scale\n{\n    return 3 * x;\n}\n"
    assert b.code_text(src) == b.code_text(commented)
    assert b.code_text(src) != b.code_text(changed)


def test_traffic_record_is_well_formed():
    # a record whose hash no longer matches is legitimate (the bench then reports null
    # traffic until the next capture); its fields must still be usable
    import json
    b = _bench()
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for name, r in rec.items():
        assert r["bytes_per_field"] > 0, name
        assert len(r["src_hash"]) == 16 and r["sources"], name
        b.src_hash(r["sources"])   # every listed source exists and hashes
