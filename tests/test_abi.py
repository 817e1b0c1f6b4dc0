"""The C-ABI library loads and exports every entry point include/kete.h
declares, and the binding's struct layouts match the header (no GPU calls)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kete.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_2509_04666_gb300 import build as B
    return B.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(kete_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_three_paper_calls():
    names = declared_functions()
    for required in ("kete_load_ephem", "kete_propagate", "kete_fov_check"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = C.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (kete_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_exports_match_header():
    from paper_2509_04666_gb300 import kete
    assert sorted(kete.EXPORTS) == declared_functions()


def test_struct_layouts_match_header(tmp_path):
    from paper_2509_04666_gb300 import kete, workloads as W
    prog = tmp_path / "sz.c"
    prog.write_text('#include "kete.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(kete_force_model),'
                    ' sizeof(kete_frame), sizeof(kete_survey_opts), sizeof(kete_hit),'
                    ' sizeof(kete_stats), offsetof(kete_frame, normals)); printf("%zu %zu %zu\\n",'
                    ' sizeof(kete_obs), sizeof(kete_mag_params), sizeof(kete_nongrav));'
                    ' return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    fm, fr, so, hit, stats, noff, ob, mg, ng = map(int,
                                                   subprocess.check_output([str(exe)]).split())
    assert fm == C.sizeof(kete.ForceModel)
    assert so == C.sizeof(kete.SurveyOpts)
    assert stats == C.sizeof(kete.Stats)
    assert fr == W.FRAME_DTYPE.itemsize == 128
    assert noff == W.FRAME_DTYPE.fields["normals"][1]
    assert hit == 32
    assert ob == W.OBS_DTYPE.itemsize == 48
    assert mg == W.MAG_DTYPE.itemsize == 24
    assert ng == W.NONGRAV_DTYPE.itemsize == 80


def test_force_model_defaults_without_gpu(libpath):
    from paper_2509_04666_gb300 import kete
    fm = kete.force_model()
    assert fm.body_mask == 0x1FF and fm.gr_mask == 0x29 and fm.j2_mask == 0x21
    assert fm.max_iter == 12 and fm.eps == 1e-9 and fm.safety == 0.25 and fm.eps_pc == 1e-10
    o = kete.survey_opts()
    assert o.batch_span == 3.0 and o.twobody_max == 1.5


def test_force_model_nongrav_argument():
    """The binding takes per-body non-gravitational terms only as a CUDA
    float64 [n, 10] tensor, and checks its rows against the call's bodies."""
    torch = pytest.importorskip("torch")
    from paper_2509_04666_gb300 import kete
    with pytest.raises(TypeError):
        kete.force_model(nongrav=torch.zeros(3, 10, dtype=torch.float64))
    with pytest.raises(TypeError):
        kete.force_model(nongrav=np.zeros((3, 10)))
    fm = kete.force_model(nongrav=None)
    assert not fm.nongrav
    kete._check_nongrav(fm, 5)


def test_nongrav_records_to_rows():
    torch = pytest.importorskip("torch")
    from paper_2509_04666_gb300 import kete, workloads as W
    ng = W.nongrav_params(np.array([3, 0, 0, 3, 1]), dust_frac=1.0, yarkovsky_every=2)
    rows = kete.nongrav_to_device(ng, "cpu")
    assert rows.shape == (5, 10) and rows.dtype == torch.float64
    for j, f in enumerate(kete.NONGRAV_FIELDS):
        assert np.array_equal(rows[:, j].numpy(), ng[f])
    # the row layout is kete_nongrav's: ten doubles in declaration order
    assert kete.NONGRAV_FIELDS == W.NONGRAV_DTYPE.names
