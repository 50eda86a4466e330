"""Extracts the fused red-black sweep kernel (layout, kernel, slab choice and launcher)
from the CUDA source so that tests/host_emu/fused_sweep_emu.cpp can compile it for the
host: the CUDA-only pieces (launch bounds, __global__, __restrict__, the shared-memory
declaration, 16-byte zero stores, the <<<...>>> launch) are rewritten into calls of the
harness's emulation shims. The kernel's own arithmetic and indexing are left untouched.

    python extract.py <smooth.cu> <out.inc>
"""
import re
import sys

MARK_END = ("// ---------------------------------------------------------------------------------\n"
            "// The same sweep with the plane rows staged by the TMA unit")


def strip_launch_bounds(text):
    while "__launch_bounds__(" in text:
        i = text.index("__launch_bounds__(")
        j = i + len("__launch_bounds__(")
        depth = 1
        while depth:
            depth += {"(": 1, ")": -1}.get(text[j], 0)
            j += 1
        text = text[:i] + text[j:]
    return text


def extract(src: str) -> str:
    body = src[src.index("constexpr int kSlots"):src.index(MARK_END)]
    ls = src.index("inline int fused_slabs(")
    le = src.index("\n}\n", src.index("int launch_shape(", ls)) + 3
    launch = src[ls:le]
    body = body.replace("extern __shared__ __align__(128) unsigned char smem_raw[];",
                        "unsigned char* smem_raw = emu_smem;")
    body = strip_launch_bounds(body).replace("__global__", "").replace("__restrict__", "")
    body = re.sub(r"\*\(int4\*\)(\w+) = make_int4\(0, 0, 0, 0\);", r"emu_zero16(\1);", body)
    launch = launch.replace("k_rbgs_fused<T, BX, BY><<<grid, Lay::threads, Lay::bytes, st>>>(",
                            "emu_launch<T, BX, BY>(grid, ")
    return body + "\n" + launch


if __name__ == "__main__":
    with open(sys.argv[1]) as fh:
        out = extract(fh.read())
    with open(sys.argv[2], "w") as fh:
        fh.write(out)
