"""C ABI checks that need no GPU: the header declares the entry points, the built
library exports every one of them, the struct layouts seen from C match the Python
binding, and creating a handle without a GPU fails loudly (no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mdeos.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mdeos_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def built_lib():
    import paper_2508_06012_gb300 as m
    return m.build()


def test_header_declares_the_boundary():
    fns = declared_functions()
    for f in ("mdeos_create", "mdeos_submit", "mdeos_poll", "mdeos_destroy", "mdeos_last_error"):
        assert f in fns


def test_library_exports_every_declared_symbol(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mdeos_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    import paper_2508_06012_gb300 as m
    assert set(m.EXPORTED) == set(declared_functions())


def test_struct_layout_matches_binding(tmp_path):
    import paper_2508_06012_gb300 as m
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "mdeos.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(mdeos_config), sizeof(mdeos_request), sizeof(mdeos_result));
  printf("%zu %zu %zu %zu\n", offsetof(mdeos_result, sigma), offsetof(mdeos_result, element_id),
         offsetof(mdeos_result, status), offsetof(mdeos_request, seed));
  printf("%zu %zu %zu %zu %zu\n", sizeof(mdeos_serve_config), offsetof(mdeos_serve_config, warm),
         offsetof(mdeos_serve_config, cluster), offsetof(mdeos_serve_config, warm_bytes),
         sizeof(mdeos_served));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    a, b, c = subprocess.run([str(exe)], capture_output=True, text=True,
                             check=True).stdout.split("\n")[:3]
    sizes = [int(v) for v in a.split()]
    offs = [int(v) for v in b.split()]
    assert sizes == [ctypes.sizeof(m.mdeos_config), ctypes.sizeof(m.mdeos_request),
                     ctypes.sizeof(m.mdeos_result)]
    assert offs == [m.mdeos_result.sigma.offset, m.mdeos_result.element_id.offset,
                    m.mdeos_result.status.offset, m.mdeos_request.seed.offset]
    serve = [int(v) for v in c.split()]
    assert serve == [ctypes.sizeof(m.mdeos_serve_config), m.mdeos_serve_config.warm.offset,
                     m.mdeos_serve_config.cluster.offset, m.mdeos_serve_config.warm_bytes.offset,
                     m.SERVED_DTYPE.itemsize]


def test_create_without_gpu_fails_loudly(built_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2508_06012_gb300 as m
    with pytest.raises(m.MdeosError) as ei:
        m.mdeos_create()
    assert ei.value.status == m.MDEOS_ECUDA


def test_invalid_config_rejected_before_device(built_lib):
    import paper_2508_06012_gb300 as m
    cfg = m.mdeos_config_default(dt=-1.0)
    with pytest.raises(m.MdeosError) as ei:
        m.mdeos_create(cfg)
    assert ei.value.status == m.MDEOS_EINVAL


def test_workload_generators_are_seeded():
    from paper_2508_06012_gb300 import workloads as w
    a, b = w.uneven_batch(nbox=64), w.uneven_batch(nbox=64)
    assert a == b
    assert {r["natoms"] for r in w.uneven_batch(nbox=4096)} == {4 * n ** 3 for n in range(3, 11)}
    assert all(0.3 <= r["rho"] <= 1.2 and 0.7 <= r["T"] <= 3.0 for r in a)
    c1 = w.small_queries()
    assert len(c1) == 16 and all(r["natoms"] == 256 for r in c1)
    assert len({r["seed"] for r in w.uneven_batch(nbox=4096)}) == 4096
