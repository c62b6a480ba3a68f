"""Compile the plain-C example against include/cddt.h and the in-tree
libcddt.so (gcc, the CUDA runtime for device memory).  Returns the binary's
path."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def build_example(out_dir: str) -> str:
    from paper_1705_01167_gb300 import build
    lib = build.build()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = os.path.join(out_dir, "cddt_example")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Werror", f"-I{os.path.join(ROOT, 'include')}",
           f"-I{os.path.join(cuda, 'include')}", os.path.join(HERE, "cddt_example.c"), "-o", exe,
           f"-L{os.path.dirname(lib)}", "-lcddt", f"-Wl,-rpath,{os.path.dirname(lib)}",
           f"-L{os.path.join(cuda, 'lib64')}", "-lcudart", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("gcc failed on the C example:\n" + r.stderr)
    return exe
