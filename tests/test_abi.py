"""The C ABI library builds, loads and exports what include/sp2.h declares
(CPU only: no compute call is made here)."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sp2.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2409_17033_gb300 import _lib
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sp2_density", "sp2_response", "sp2_susceptibility", "response_contract",
                     "sp2_adjoint", "sp2_create", "sp2_destroy", "sp2_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    from paper_2409_17033_gb300 import _lib
    assert set(_lib.EXPORTS) >= set(declared_functions())


def test_nm_shows_c_linkage(lib):
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    from paper_2409_17033_gb300 import _lib
    out = subprocess.run([nm, "-D", "--defined-only", _lib.LIB_PATH], capture_output=True,
                         text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in declared_functions():
        assert name in syms, f"{name} not exported with C linkage"


def test_struct_layout_matches_c(tmp_path, lib):
    """sizeof/offsetof of sp2_opts, sp2_info and sp2_scf_opts from a C compiler
    agree with the ctypes mirror used by the binding."""
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2409_17033_gb300 import _lib
    probe = tmp_path / "probe.c"
    fields_o = [f for f, _ in _lib.Opts._fields_]
    fields_i = [f for f, _ in _lib.Info._fields_]
    fields_s = [f for f, _ in _lib.ScfOpts._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){",
             'printf("%zu %zu %zu\\n", sizeof(sp2_opts), sizeof(sp2_info), sizeof(sp2_scf_opts));']
    for f in fields_o:
        lines.append(f'printf("%zu\\n", offsetof(sp2_opts, {f}));')
    for f in fields_i:
        lines.append(f'printf("%zu\\n", offsetof(sp2_info, {f}));')
    for f in fields_s:
        lines.append(f'printf("%zu\\n", offsetof(sp2_scf_opts, {f}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([gcc, str(probe), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals[0] == C.sizeof(_lib.Opts)
    assert vals[1] == C.sizeof(_lib.Info)
    assert vals[2] == C.sizeof(_lib.ScfOpts)
    offs = vals[3:]
    no, ni = len(fields_o), len(fields_i)
    for f, off in zip(fields_o, offs[:no]):
        assert getattr(_lib.Opts, f).offset == off, f
    for f, off in zip(fields_i, offs[no:no + ni]):
        assert getattr(_lib.Info, f).offset == off, f
    for f, off in zip(fields_s, offs[no + ni:]):
        assert getattr(_lib.ScfOpts, f).offset == off, f
    assert len(offs) == no + ni + len(fields_s)


def test_default_opts_host_only(lib):
    """sp2_default_opts is pure host code: callable without a GPU."""
    from paper_2409_17033_gb300 import _lib
    o = _lib.Opts()
    lib.sp2_default_opts(C.byref(o))
    assert o.mode == _lib.MODE_FP32
    assert o.max_iter == 100 and o.min_iter == 4 and o.ckpt_k == 4
    assert o.floor_gate == pytest.approx(0.03)
    assert o.fixed_m == 0 and not o.sigma_in


def test_null_handle_is_rejected(lib):
    """Argument validation happens before any CUDA call."""
    from paper_2409_17033_gb300 import _lib
    assert lib.sp2_destroy(None) == _lib.EINVAL
    assert lib.sp2_density(None, None, 4, 0, 2.0, None, None, None) == _lib.EINVAL
    assert lib.sp2_create(None, None, 0) == _lib.EINVAL


def test_make_opts_host_only(lib):
    """The binding's option marshalling is host code: the automatic checkpoint
    interval, the mode names (BF16X3 included) and the branch array."""
    from paper_2409_17033_gb300 import _lib, api
    o, keep = api.make_opts("bf16x3", ckpt_k="auto", sigma=[1, -1, 1])
    assert o.mode == _lib.MODE_BF16X3 == 4
    assert o.ckpt_k == _lib.CKPT_AUTO == -1
    assert o.fixed_m == 3 and [o.sigma_in[i] for i in range(3)] == [1, -1, 1]
    o2, _ = api.make_opts("fp16x2", ckpt_k=1, bounds=(-2.0, 3.0))
    assert o2.ckpt_k == 1 and (o2.eps_min, o2.eps_max) == (-2.0, 3.0)


def test_info_dict_fields(lib):
    """sp2_info exposes the checkpoint interval used and the refinement /
    Newton-Schulz iteration field to Python."""
    from paper_2409_17033_gb300 import _lib
    d = _lib.Info().to_dict()
    assert "ckpt_k" in d and "refine_iter" in d


def test_mode_constants_match_the_header(tmp_path, lib):
    """The binding's mode numbers and SP2_DEFAULT_TAIL_F are the header's."""
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2409_17033_gb300 import _lib
    probe = tmp_path / "modes.c"
    names = ["SP2_MODE_FP64", "SP2_MODE_FP32", "SP2_MODE_BF16X2", "SP2_MODE_FP16X2",
             "SP2_MODE_BF16X3", "SP2_MODE_BF16_TAIL"]
    lines = ['#include <stdio.h>', f'#include "{HEADER}"', "int main(void){"]
    lines += [f'printf("%d\\n", (int){n});' for n in names]
    lines += ['printf("%.17g\\n", (double)SP2_DEFAULT_TAIL_F);', "return 0;}"]
    probe.write_text("\n".join(lines))
    exe = tmp_path / "modes"
    subprocess.run([gcc, str(probe), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out[:-1]]
    assert got == [_lib.MODE_FP64, _lib.MODE_FP32, _lib.MODE_BF16X2, _lib.MODE_FP16X2,
                   _lib.MODE_BF16X3, _lib.MODE_BF16_TAIL]
    assert [_lib.MODES[k] for k in ("fp64", "fp32", "bf16x2", "fp16x2", "bf16x3", "bf16_tail")] == got
    assert float(out[-1]) == _lib.DEFAULT_TAIL_F
