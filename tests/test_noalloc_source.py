"""residual_noalloc allocates nothing: neither its translation unit nor the operator set-up and
launch code it calls (kernels_impl.cuh: prepare_op, launch_op) names a device allocation or
release routine. A CPU check of the sources; the GPU test checks free device memory."""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1904_03057_gb300", "csrc")
ALLOC = re.compile(r"\b(cudaMalloc\w*|cudaFree\w*|cuMemAlloc\w*|cuMemFree\w*|malloc|new\s)")


def _code(path):
    text = open(path).read()
    text = re.sub(r"//[^\n]*", "", text)          # comments may mention allocation
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def test_noalloc_path_names_no_allocation():
    for name in ("noalloc.cu", "kernels_impl.cuh", "op_generic.cuh"):
        hits = ALLOC.findall(_code(os.path.join(CSRC, name)))
        assert not hits, (name, hits)
