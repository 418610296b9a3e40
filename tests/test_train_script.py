"""Host logic of the bracket-training script.  CPU only."""
import struct

import pytest


def test_checkpoint_step_reads_the_header(tmp_path):
    import __graft_entry__
    __graft_entry__.build()          # the package loads the library on import
    from paper_1104_2732_gb300 import train_bracket as tb
    p = tmp_path / "m.bin"
    p.write_bytes(b"GBSBRKT1" + struct.pack("<5I", 1, 36, 64, 2, 6914) + struct.pack("<Q", 12345) + b"\0" * 16)
    assert tb.checkpoint_step(str(p)) == 12345
    q = tmp_path / "bad.bin"
    q.write_bytes(b"NOTAMODL" + b"\0" * 40)
    with pytest.raises(ValueError):
        tb.checkpoint_step(str(q))
    r = tmp_path / "short.bin"
    r.write_bytes(b"GBSBRKT1")
    with pytest.raises(ValueError):
        tb.checkpoint_step(str(r))
