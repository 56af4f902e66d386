"""The planted-mistake sweep's machinery (tests/oracle_mutation_sweep.py) on one entry:
an unmodified copy of the oracle built to a temporary library passes the pin it targets,
and the copy with the mistake planted fails it."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def _pin_passes(so_path, pin):
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins_dvm.py", "-q", "-k", pin,
                        "-p", "no:cacheprovider"], cwd=ROOT, capture_output=True, text=True,
                       env=dict(os.environ, SDUGKS_ORACLE_LIB=so_path))
    return r.returncode == 0


def test_sweep_plants_a_mistake_the_pin_catches(tmp_path):
    import oracle
    import oracle_mutation_sweep as sweep
    (what, pins, old, new, which), = [m for m in sweep.MUTATIONS if m[0] == "rarefied: relaxation rate dt/(2 tau)"]
    with open(os.path.join(ROOT, "oracle", "sdugks_oracle.c")) as fh:
        src = fh.read()
    i = src.rindex(old)
    clean, planted = tmp_path / "clean.c", tmp_path / "planted.c"
    clean.write_text(src)
    planted.write_text(src[:i] + new + src[i + len(old):])
    so_clean = oracle.compile_library(str(clean), str(tmp_path / "clean.so"))
    so_planted = oracle.compile_library(str(planted), str(tmp_path / "planted.so"))
    assert _pin_passes(so_clean, "relaxes_at_the_bgk_rate")
    assert not _pin_passes(so_planted, "relaxes_at_the_bgk_rate")
