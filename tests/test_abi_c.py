"""The C ABI from C: include/pdf.h compiles as strict C99, a C program links against the library
and calls it without a GPU (defaults, argument rejection), and every field of the public structs
sits at the same offset in C as in the Python binding's ctypes layouts."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2602_13805_gb300 import build, pdf
    build.build()
    pdf.load()
    return os.path.join(ROOT, "paper_2602_13805_gb300")


def _program(structs):
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pdf.h"', "int main(void) {",
             "  pdf_config c;", "  pdf_solve_opts o;", "  pdf_config_default(&c);", "  pdf_solve_opts_default(&o);",
             '  printf("defaults %d %g %d %g\\n", o.iters, o.lr, o.use_graph, c.beta_re);',
             '  printf("reject %d %d\\n", (int)pdf_solve(NULL, &o, NULL, NULL, NULL, NULL, NULL),'
             " (int)pdf_loss_grad(NULL, NULL, NULL, NULL, NULL));"]
    for cname, cls in structs:
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("off {cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


def test_header_is_c99_and_layouts_match_binding(built, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2602_13805_gb300 import pdf
    structs = [("pdf_config", pdf.pdf_config), ("pdf_solve_opts", pdf.pdf_solve_opts),
               ("pdf_solve_report", pdf.pdf_solve_report)]
    src = tmp_path / "abi.c"
    src.write_text(_program(structs))
    exe = tmp_path / "abi"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", built, "-lpdf", f"-Wl,-rpath,{built}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    kv = {}
    for line in out:
        key, _, val = line.rpartition(" ")
        kv[key] = val
    assert out[0] == "defaults 300 0.01 3 6"
    assert out[1] == "reject -1 -1"
    for cname, cls in structs:
        assert int(kv[f"size {cname}"]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(kv[f"off {cname}.{fname}"]) == getattr(cls, fname).offset, f"{cname}.{fname}"
