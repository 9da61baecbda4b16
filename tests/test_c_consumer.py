"""libfbcc from plain C: include/fbcc.h is strict C99 on its own, and a C program
(tests/c/solve_from_c.c) that uses only the header and the CUDA runtime compiles
and links against the library here; on a GPU its results, from two solves in a
row, equal the oracle's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2301_01356_gb300 import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c", "solve_from_c.c")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    return cc


def _libdir():
    from paper_2301_01356_gb300 import build
    return os.path.dirname(build.build_libfbcc())


def _compile(tmp_path) -> str:
    exe = str(tmp_path / "solve_from_c")
    cudalib = next((d for d in (os.path.join(CUDA, "lib64"), os.path.join(CUDA, "lib"),
                                os.path.join(CUDA, "targets", "sbsa-linux", "lib")) if os.path.isdir(d)), None)
    if cudalib is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("no CUDA toolkit headers and runtime library")
    lib = _libdir()
    subprocess.run([_cc(), "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(CUDA, "include"), SRC, "-L", lib, "-lfbcc", "-L", cudalib, "-lcudart",
                    f"-Wl,-rpath,{lib}", f"-Wl,-rpath,{cudalib}", "-o", exe], check=True)
    return exe


def test_header_is_strict_c99(tmp_path):
    src = tmp_path / "h.c"
    src.write_text('#include "fbcc.h"\nint main(void) { return fbcc_status_string(FBCC_OK) == 0; }\n')
    subprocess.run([_cc(), "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                    os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "h.o")], check=True)


def test_c_program_compiles_and_links(tmp_path):
    assert os.path.exists(_compile(tmp_path))


def _read_out(path, n, nnz):
    raw = open(path, "rb").read()
    outs, at = [], 0
    for _ in range(2):
        head = np.frombuffer(raw, np.int64, 5, at)
        at += 40
        nb = int(head[0])
        eb = np.frombuffer(raw, np.int32, nnz, at); at += 4 * nnz
        bh = np.frombuffer(raw, np.int32, nb, at); at += 4 * nb
        ap = np.frombuffer(raw, np.uint8, n, at); at += n
        br = np.frombuffer(raw, np.uint8, nnz, at); at += nnz
        outs.append({"n_bcc": nb, "n_ap": int(head[1]), "n_bridge": int(head[2]), "n_cc": int(head[3]),
                     "device_status": int(head[4]), "edge_bcc": eb, "bcc_head": bh, "is_ap": ap, "is_bridge": br})
    assert at == len(raw)
    return outs


@pytest.mark.gpu
def test_c_program_matches_oracle(tmp_path, oracle):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _compile(tmp_path)
    for g in (gg.cycles_chain_exact([3, 4, 5, 6], 2), gg.grid(60, 50, p=0.62, seed=3), gg.rmat(12, 8, seed=4),
              gg.from_edges(4, [], [])):
        gpath, opath = tmp_path / "g.bin", tmp_path / "o.bin"
        with open(gpath, "wb") as f:
            f.write(np.array([g.n, g.nnz], np.int64).tobytes())
            f.write(g.offsets.astype(np.int32).tobytes())
            f.write(g.adj.astype(np.int32).tobytes())
        subprocess.run([exe, str(gpath), str(opath)], check=True)
        exp = oracle.solve(g.offsets, g.adj)
        for got in _read_out(opath, g.n, g.nnz):
            assert got["device_status"] == 0
            for k in ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge", "n_cc"):
                assert np.array_equal(np.asarray(got[k]), np.asarray(exp[k])), (g.name, k)
