"""The C-ABI library builds, loads and exports every symbol the header
declares; the ctypes structs match the header's layout (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "clsplat.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cls_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_21117_gb300 import build
    from paper_2506_21117_gb300 import _abi
    build.build()
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2506_21117_gb300 import _abi
    names = _declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_abi.SIGNATURES) == names


def test_host_only_entry_points(lib):
    from paper_2506_21117_gb300 import _abi
    assert [_abi.cls_row_stride(d) for d in range(4)] == [16, 24, 40, 64]
    assert _abi.cls_row_stride(4) == -1
    assert "sm_103a" in _abi.cls_version()
    assert _abi.cls_sort_workspace_size(1000, 47) > 0
    assert _abi.cls_lift_workspace_size(10) > 0


def test_batch_prepare_derived_fields(lib):
    from paper_2506_21117_gb300 import _abi
    from paper_2506_21117_gb300.update import make_camera
    from paper_2506_21117_gb300 import synthetic as S
    cams = S.ring_cameras(2, 4.0, 100, 70) + S.ring_cameras(1, 4.0, 32, 32)
    scenes = (_abi.ClsScene * 2)()
    scenes[0].n, scenes[0].row_stride, scenes[0].sh_degree = 1000, 64, 3
    scenes[0].n_active, scenes[0].first_view, scenes[0].n_views = 10, 0, 2
    scenes[1].n, scenes[1].row_stride, scenes[1].sh_degree = 50, 16, 0
    scenes[1].n_active, scenes[1].first_view, scenes[1].n_views = 50, 2, 1
    views = (_abi.ClsView * 3)()
    for j, (cam, s) in enumerate(zip(cams, [0, 0, 1])):
        views[j].cam = make_camera(cam)
        views[j].scene = s
    info = _abi.ClsBatchInfo()
    assert _abi.cls_batch_prepare(scenes, views, info) == 0
    assert [views[j].tile_base for j in range(3)] == [0, 35, 70]
    assert [views[j].rec_base for j in range(3)] == [0, 1000, 2000]
    assert [views[j].g2_base for j in range(3)] == [0, 10, 20]
    assert [views[j].pix_base for j in range(3)] == [0, 7000, 14000]
    assert scenes[1].grad_base == 10
    assert info.total_tiles == 74 and info.total_records == 2050
    assert info.key_bits == 32 + 7
    assert abs(views[2].loss_scale * (3 * 32 * 32) - 1.0) < 1e-7
    views[2].scene = 0  # view outside its scene's range
    assert _abi.cls_batch_prepare(scenes, views, info) == _abi.CLS_ERR_INVALID_ARG


def test_struct_layout_matches_header():
    """Compile a host C program against the header and compare sizeof/offsetof
    with the ctypes mirrors."""
    from paper_2506_21117_gb300 import _abi
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "clsplat.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(ClsCamera), sizeof(ClsScene), sizeof(ClsView),
         sizeof(ClsBatchInfo), sizeof(ClsProjected));
  printf("%zu %zu %zu %zu %zu\n", offsetof(ClsView, scene), offsetof(ClsView, rec_base),
         offsetof(ClsView, loss_scale), offsetof(ClsScene, grad_base),
         offsetof(ClsBatchInfo, total_tiles));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), src, "-o", exe],
                       check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [C.sizeof(t) for t in (_abi.ClsCamera, _abi.ClsScene, _abi.ClsView,
                                   _abi.ClsBatchInfo, _abi.ClsProjected)]
    offs = [_abi.ClsView.scene.offset, _abi.ClsView.rec_base.offset,
            _abi.ClsView.loss_scale.offset, _abi.ClsScene.grad_base.offset,
            _abi.ClsBatchInfo.total_tiles.offset]
    assert [int(x) for x in out] == sizes + offs
