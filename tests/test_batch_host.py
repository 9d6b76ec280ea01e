"""Host logic of the batched module: the HLF_SPIN_LIMIT override."""

import pytest

from paper_2103_00693_gb300 import batch


def test_spin_limit_env_parsing(monkeypatch):
    monkeypatch.delenv("HLF_SPIN_LIMIT", raising=False)
    assert batch.spin_limit_from_env() is None
    monkeypatch.setenv("HLF_SPIN_LIMIT", "0x100")
    assert batch.spin_limit_from_env() == 256
    monkeypatch.setenv("HLF_SPIN_LIMIT", "1000")
    assert batch.spin_limit_from_env() == 1000
    for bad in ("0", "-5", str(1 << 32)):
        monkeypatch.setenv("HLF_SPIN_LIMIT", bad)
        with pytest.raises(ValueError):
            batch.spin_limit_from_env()
