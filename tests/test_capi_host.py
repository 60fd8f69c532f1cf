"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every symbol that include/*.h declares, and rejects malformed
problems with MRPOP_EINVAL before touching the device."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2609_30644_gb300 import build as B
    B.build()
    import paper_2609_30644_gb300 as m
    return m


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(mrpop_[a-z0-9_]+)\s*\(", txt))
    return names


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("mrpop_create_problem", "mrpop_validate_edges", "mrpop_nearest",
              "mrpop_neighbors", "mrpop_path_cost", "mrpop_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(capi):
    lib = C.CDLL(capi.library_path)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(capi.EXPORTS) == declared_symbols()


def _scene():
    from paper_2609_30644_gb300 import synth
    return synth.planar_pair_scene(0)


@pytest.mark.parametrize("mutate,msg", [
    (lambda s: s.robots[0].__setattr__("dof", 0), "dof"),
    (lambda s: s.robots[0].__setattr__("dof", 17), "dof"),
    (lambda s: s.robots[0].sphere_link.__setitem__(0, 2), "non-decreasing"),
    (lambda s: s.robots[0].sphere_xyzr.__setitem__((0, 3), -1.0), "radius"),
    (lambda s: s.obs_spheres.__setitem__((0, 3), np.nan), "non-finite"),
    (lambda s: s.robots[1].base.__setitem__(3, np.inf), "non-finite"),
    (lambda s: s.robots[0].base.__setitem__(slice(8, 11), [0.0, 0.0, -1.0]), "proper rotation"),
    (lambda s: s.robots[0].base.__setitem__(0, 1.5), "proper rotation"),
])
def test_create_rejects_malformed(capi, mutate, msg):
    s = _scene()
    mutate(s)
    with pytest.raises(capi.MrpopError) as ei:
        capi.Problem(s)
    assert ei.value.status == 1 and msg in str(ei.value)


def test_create_rejects_too_many_spheres_per_link(capi):
    from paper_2609_30644_gb300 import synth
    rb = synth.planar_arm(np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32),
                          spheres_per_link=17)
    s = synth.Scene([rb], np.zeros((0, 4), np.float32), np.zeros((0, 15), np.float32))
    with pytest.raises(capi.MrpopError) as ei:
        capi.Problem(s)
    assert ei.value.status == 1


def test_create_rejects_bad_config(capi):
    with pytest.raises(capi.MrpopError) as ei:
        capi.Problem(_scene(), resolution=0.0)
    assert ei.value.status == 1
    with pytest.raises(capi.MrpopError):
        capi.Problem(_scene(), margin=-1.0)


def test_create_rejects_bad_self_mask(capi):
    """A self-collision mask bit at or above its own link is malformed; with
    self-collision off the mask is ignored."""
    import dataclasses
    s = _scene()
    s.robots[0] = dataclasses.replace(s.robots[0], self_mask=np.array([0, 2, 1], np.uint16))
    with pytest.raises(capi.MrpopError) as ei:
        capi.Problem(s, self_collision=True)
    assert ei.value.status == 1 and "self_mask" in str(ei.value)
    with pytest.raises(capi.MrpopError) as ei:   # valid tables: fails only at the device
        capi.Problem(s, self_collision=False)
    assert "self_mask" not in str(ei.value)


def test_nearest_rejects_bad_dim(capi):
    lib = capi.lib
    st = lib.mrpop_nearest(None, 0, 0, 0, None, None, 1, None, None)
    assert st == 1 and b"dim" in lib.mrpop_last_error()
    st = lib.mrpop_nearest(None, 10, 5, 3, None, None, 1, None, None)   # ld < N
    assert st == 1
    assert lib.mrpop_nearest(None, 0, 0, 3, None, None, 0, None, None) == 0  # Q = 0: no-op


def test_autotune_cache_save_load_roundtrip(capi, tmp_path):
    """The tuned-launch cache is host data: entries loaded from a file come
    back out of a save unchanged, later loads replace keys, a malformed line
    is refused with MRPOP_EINVAL, and clearing empties it."""
    src = tmp_path / "in.txt"
    src.write_text("# comment\n"
                   "validate sm_00 K=2 L=14 S=120 NS=32 NC=32 spl=9 self=0 = 4 0 0 1\n"
                   "nearest sm_00 dim=14 N=2^14 Q=2^16 filter=0 = 8\n")
    capi.autotune_cache_clear()
    capi.autotune_cache_load(str(src))
    capi.autotune_cache_load(str(src))                 # idempotent
    out = tmp_path / "out.txt"
    capi.autotune_cache_save(str(out))
    entries = {l.split(" = ")[0]: l.split(" = ")[1] for l in out.read_text().splitlines()
               if l and not l.startswith("#")}
    assert entries == {"validate sm_00 K=2 L=14 S=120 NS=32 NC=32 spl=9 self=0": "4 0 0 1",
                       "nearest sm_00 dim=14 N=2^14 Q=2^16 filter=0": "8"}
    upd = tmp_path / "upd.txt"
    upd.write_text("nearest sm_00 dim=14 N=2^14 Q=2^16 filter=0 = 2\n")
    capi.autotune_cache_load(str(upd))
    capi.autotune_cache_save(str(out))
    assert "nearest sm_00 dim=14 N=2^14 Q=2^16 filter=0 = 2" in out.read_text()
    bad = tmp_path / "bad.txt"
    bad.write_text("no separator here\n")
    with pytest.raises(capi.MrpopError) as e:
        capi.autotune_cache_load(str(bad))
    assert e.value.status == 1
    bad.write_text("k = 1 x\n")
    with pytest.raises(capi.MrpopError):
        capi.autotune_cache_load(str(bad))
    capi.autotune_cache_clear()
    capi.autotune_cache_save(str(out))
    assert [l for l in out.read_text().splitlines() if not l.startswith("#")] == []
