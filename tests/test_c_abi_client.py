"""The C ABI used from plain C99: tests/c_abi_client.c includes only include/ajf.h, links only
libajf.so, and drives loading, noise, planning, the plan check and the documented error paths on a
host-only context. Its plan figures must equal the Python binding's for the same circuit, which
shows that the binding only marshals arguments."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2103_11595_gb300 import ajf
from paper_2103_11595_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    import __graft_entry__
    __graft_entry__.build()
    libdir = os.path.dirname(ajf.LIB_PATH)
    exe = str(tmp_path_factory.mktemp("c_client") / "ajf_c_client")
    subprocess.run(["gcc", "-std=c99", "-O1", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_abi_client.c"),
                    "-L", libdir, "-lajf", f"-Wl,-rpath,{libdir}", "-lm", "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return dict(line.split(" ", 1) for line in out.strip().splitlines())


def test_c_client_runs_every_call(client):
    assert client["done"] == "1"
    assert "not trace preserving" in client["last_error"]


def test_c_client_plans_equal_the_binding(client):
    r = 1 / np.sqrt(2)
    H = np.array([[r, r], [r, -r]], dtype=np.complex128)
    inst = W.Instance(2, [W.Gate((0,), H), W.Gate((0, 1), W.CX)],
                      [W.Noise(0, (0,), W.depolarising(0.01), "dep")])
    for alg in (1, 2):
        with ajf.Context(-1) as c:
            ajf.load_instance(c.handle, inst)
            info = ajf.ajf_plan(c.handle, alg, trials=4)
        assert int(client[f"alg{alg}_leaves"]) == info["n_leaves"]
        assert int(client[f"alg{alg}_open_bits"]) == info["n_open_bits"]
        assert int(client[f"alg{alg}_width"]) == info["width"]
        assert float(client[f"alg{alg}_cmacs"]) == info["cmacs"]
        assert int(client[f"alg{alg}_units"]) == 1
    assert int(client["alg1_open_bits"]) == 2  # four Kraus operators: one 2-bit open index
