"""There is no CPU fallback: without the CUDA library, or without a GPU, the
binding raises instead of computing anything on the host."""
import pytest

torch = pytest.importorskip("torch")


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_2112_06396_gb300 import ckks

    monkeypatch.setattr(ckks, "_lib", None)
    monkeypatch.setattr(ckks._build, "LIB", str(tmp_path / "libckks_ks.so"))
    with pytest.raises(ckks.CkksError, match="missing"):
        ckks.lib()
    with pytest.raises(ckks.CkksError):
        ckks.ckks_gen_primes(50, 12, 9)
    with pytest.raises(ckks.CkksError):
        ckks.Context(12, [1125899906826241], [1125899906629633], 1)


def test_context_without_a_gpu_raises():
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2112_06396_gb300 import build, ckks

    try:
        build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    primes = ckks.ckks_gen_primes(50, 12, 9)  # host-only entry point
    with pytest.raises(ckks.CkksError) as err:
        ckks.Context(12, primes[:6], primes[6:], 2)
    assert err.value.code == ckks.CKKS_ECUDA
