"""The gate checkpoint file format on CPU: a round trip keeps every tensor and
the step count bit for bit; a flipped byte, a truncated file or a foreign file
is refused."""
import pytest

torch = pytest.importorskip("torch")


def _ckpt():
    g = torch.Generator().manual_seed(7)
    return {"t": 12, "params": torch.randn(81, generator=g), "m1p": torch.randn(81, generator=g),
            "m2p": torch.rand(81, generator=g), "emb": torch.randn(50, 128, generator=g),
            "m1e": torch.zeros(50, 128), "m2e": torch.full((50, 128), 1e-8)}


def test_round_trip_is_bit_exact(tmp_path):
    from paper_2602_17330_gb300 import train

    c = _ckpt()
    path = str(tmp_path / "gate.ckpt")
    train.write_checkpoint(path, c)
    back = train.read_checkpoint(path)
    assert back["t"] == 12 and set(back) == set(c)
    for k, v in c.items():
        if torch.is_tensor(v):
            assert back[k].dtype == v.dtype and back[k].shape == v.shape
            assert torch.equal(back[k].view(torch.int32), v.view(torch.int32)), k


@pytest.mark.parametrize("damage", ["flip", "truncate", "foreign"])
def test_damaged_files_are_refused(tmp_path, damage):
    from paper_2602_17330_gb300 import train

    path = tmp_path / "gate.ckpt"
    train.write_checkpoint(str(path), _ckpt())
    raw = bytearray(path.read_bytes())
    if damage == "flip":
        raw[len(raw) // 2] ^= 0x40
    elif damage == "truncate":
        raw = raw[:-100]
    else:
        raw = bytearray(b"PK\x03\x04" + bytes(200))
    path.write_bytes(bytes(raw))
    with pytest.raises(ValueError):
        train.read_checkpoint(str(path))
