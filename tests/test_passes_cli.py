"""The per-level pass timer's command line parses without a GPU (the GPU work
starts only after the arguments are read)."""

import pytest

from paper_1705_06266_gb300 import passes


def test_help_exits_cleanly(capsys):
    with pytest.raises(SystemExit) as e:
        passes.main(["--help"])
    assert e.value.code == 0
    out = capsys.readouterr().out
    for flag in ("--rmat", "--workload", "--complete", "--levels", "--batch", "--opt", "--setups"):
        assert flag in out


def test_sources_are_exclusive():
    with pytest.raises(SystemExit):
        passes.main(["--rmat", "20", "--workload", "rmat_20"])
