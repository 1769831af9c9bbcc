"""GPU: the C ABI from plain C (examples/abi_demo.c), without Python in the
loop: keygen, encrypt, mul_relin, mod_to_bits, bits_to_mod, decrypt and
bfhe_check, checked against plain arithmetic by the program itself."""

import subprocess

import pytest

from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_plain_c_program_through_the_abi():
    need_gpu()
    from paper_2204_12201_gb300 import build
    exe, _ = build.build_demo()
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "abi demo ok" in r.stdout
