"""The product path has no CPU fallback: without the compiled library every entry point raises,
and the package never imports the oracle."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2602_13805_gb300")


def test_missing_library_raises():
    code = (
        "import sys\n"
        "from paper_2602_13805_gb300 import pdf\n"
        "pdf.load.__defaults__ = ('/nonexistent/libpdf.so',)     # as if the build had not run\n"
        "try:\n"
        "    pdf.load('/nonexistent/libpdf.so')\n"
        "except pdf.PDFError as e:\n"
        "    assert 'missing' in str(e), e\n"
        "else:\n"
        "    sys.exit('load did not raise')\n"
        "for call in (lambda: pdf.pdf_launch_count(), lambda: pdf.pdf_fp32_fma_peak(1)):\n"
        "    try:\n"
        "        call()\n"
        "    except pdf.PDFError:\n"
        "        pass\n"
        "    else:\n"
        "        sys.exit('an entry point ran without the library')\n"
    )
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr


def test_package_never_imports_the_oracle():
    pat = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)", re.M)
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(".py"):
                src = open(os.path.join(dirpath, f)).read()
                assert not pat.search(src), os.path.join(dirpath, f)


def test_oracle_never_imports_the_package():
    pat = re.compile(r"paper_2602_13805_gb300|libpdf")
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        if f.endswith(".py"):
            assert not pat.search(open(os.path.join(odir, f)).read()), f
