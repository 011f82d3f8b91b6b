"""The C-ABI library loads on a machine without a GPU and exports what
include/lgt.h declares; host-side argument checks run without a device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lgt.h")


@pytest.fixture(scope="module")
def lgt():
    from paper_1305_3440_gb300 import build
    build.build()
    from paper_1305_3440_gb300 import lgt as mod
    return mod


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^LGT_API[^(]*?\b(lgt_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lgt):
    names = declared_symbols()
    assert len(names) >= 20
    lib = ctypes.CDLL(lgt.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in lgt.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", lgt.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lgt_\w+)$", out, flags=re.M))
    assert exported == set(names), f"exported but undeclared: {exported - set(names)}"


def test_struct_layout_matches_header(lgt, tmp_path):
    """sizeof/offsetof from a C program compiled against lgt.h equal the binding's."""
    src = tmp_path / "probe.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "lgt.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(lgt_params), offsetof(lgt_params, omega),
         offsetof(lgt_params, theta_tol), offsetof(lgt_params, block_size), sizeof(lgt_result));
  printf("%zu %zu %zu\\n", offsetof(lgt_result, sweeps_bulk), offsetof(lgt_result, status), sizeof(lgt_stats));
  return 0;
}
""")
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    a, b = subprocess.check_output([str(exe)], text=True).split("\n")[:2]
    P, R, S = lgt.lgt_params, lgt.lgt_result, lgt.lgt_stats
    assert [int(v) for v in a.split()] == [ctypes.sizeof(P), P.omega.offset, P.theta_tol.offset,
                                           P.block_size.offset, ctypes.sizeof(R)]
    assert [int(v) for v in b.split()] == [R.sweeps_bulk.offset, R.status.offset, ctypes.sizeof(S)]


def test_defaults(lgt):
    p = lgt.lgt_params_default()
    assert p.omega == 1.7 and p.theta_tol == 1e-14 and p.check_every == 10 and p.bulk == lgt.LGT_FP64
    assert list(p.dims) == [0, 0, 0, 0] and p.transform_temporal == 1


@pytest.mark.parametrize("field,value", [("dims", (8, 8, 8, 7)), ("dims", (0, 8, 8, 8)),
                                         ("omega", 2.0), ("omega", 0.9), ("check_every", 0),
                                         ("block_size", 96), ("theta_tol", 0.0), ("bulk", 7),
                                         ("launch_config", 17), ("launch_config", -1), ("sa_sweeps", -1),
                                         ("polish_algo", 2), ("polish_algo", -1), ("omega_late", 2.0), ("omega_late", 0.5),
                                         ("theta_omega", -1.0)])
def test_bad_params_rejected_before_any_device_work(lgt, field, value):
    import numpy as np
    kw = {"dims": (4, 4, 4, 4), field: value}
    p = lgt.lgt_params_default(**kw)
    links = np.zeros((4, 4, 4, 4, 4, 3, 3), np.complex128)
    with pytest.raises(lgt.LgtError) as e:
        lgt.lgt_create(p, links)
    assert e.value.status == lgt.LGT_EINVAL
    assert lgt.lgt_last_error()


def test_gauge_range_and_mag_without_annealing(lgt):
    """gauge 3 is unknown; the maximally Abelian gauge takes no annealing sweeps.
    Both are refused by the parameter check, before any device work."""
    import numpy as np
    links = np.zeros((4, 4, 4, 4, 4, 3, 3), np.complex128)
    for kw in (dict(gauge=3), dict(gauge=lgt.LGT_MAG, sa_sweeps=2)):
        with pytest.raises(lgt.LgtError) as e:
            lgt.lgt_create(lgt.lgt_params_default(dims=(4, 4, 4, 4), **kw), links)
        assert e.value.status == lgt.LGT_EINVAL


@pytest.mark.parametrize("b0,b1", [(0.0, 1.0), (2.0, 1.0), (1.0, float("inf"))])
def test_annealing_schedule_rejected(lgt, b0, b1):
    import numpy as np
    p = lgt.lgt_params_default(dims=(4, 4, 4, 4), sa_sweeps=3, sa_beta0=b0, sa_beta1=b1)
    with pytest.raises(lgt.LgtError):
        lgt.lgt_create(p, np.zeros((4, 4, 4, 4, 4, 3, 3), np.complex128))


def test_sr_probability_range(lgt):
    import numpy as np
    p = lgt.lgt_params_default(dims=(4, 4, 4, 4), algo=lgt.LGT_SR, p=1.5)
    with pytest.raises(lgt.LgtError):
        lgt.lgt_create(p, np.zeros((4, 4, 4, 4, 4, 3, 3), np.complex128))


def test_version(lgt):
    assert "sm_103a" in lgt.lgt_version()


def test_injected_allocation_failure_is_reported(lgt):
    """LGT_FAULT=alloc makes context and server creation fail with LGT_ENOMEM, with no
    device work (the failure is made on the host)."""
    import subprocess
    import sys
    code = (
        "import numpy as np\n"
        "from paper_1305_3440_gb300 import lgt\n"
        "p = lgt.lgt_params_default(dims=(4, 4, 4, 4))\n"
        "try:\n"
        "    lgt.lgt_create(p, np.zeros((4, 4, 4, 4, 4, 3, 3), np.complex128))\n"
        "except lgt.LgtError as e:\n"
        "    assert e.status == lgt.LGT_ENOMEM and 'injected' in lgt.lgt_last_error(), e\n"
        "else:\n"
        "    raise SystemExit('no failure')\n"
        "try:\n"
        "    lgt.lgt_server_create(1 << 30, 0)\n"
        "except lgt.LgtError as e:\n"
        "    assert e.status == lgt.LGT_ENOMEM\n"
        "else:\n"
        "    raise SystemExit('no failure')\n"
        "print('ok')\n")
    env = dict(os.environ, LGT_FAULT="nan,alloc", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
