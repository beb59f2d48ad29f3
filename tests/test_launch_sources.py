"""Every kernel launched with programmatic stream serialization waits first.

launch_dependent lets a kernel be scheduled while the previous kernel of
the stream is still running, which is only safe if the kernel executes
griddepcontrol.wait (griddep_wait) before it touches global memory.  This
checks the sources: every kernel handed to launch_dependent -- by name, or
through the dense launcher's `kern` pointer -- calls griddep_wait(), and
no such call sits behind a global load or store of the kernel's
arguments.  The check reads the CUDA sources as text; it needs no GPU.
"""
from __future__ import annotations

import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2606_26439_gb300", "csrc")


def _sources():
    out = {}
    for name in sorted(os.listdir(CSRC)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, name)) as f:
                out[name] = f.read()
    return out


def _kernel_body(text: str, name: str) -> str:
    """The body of `__global__ ... name(...) { ... }` (first definition)."""
    m = re.search(r"__global__[^;{]*?\b" + re.escape(name) + r"\s*\(", text, re.S)
    assert m, f"kernel {name} not found"
    i = text.index("{", m.end())
    depth = 0
    for j in range(i, len(text)):
        if text[j] == "{":
            depth += 1
        elif text[j] == "}":
            depth -= 1
            if depth == 0:
                return text[i:j + 1]
    raise AssertionError(f"unbalanced body for {name}")


def _launched_kernels(src):
    names = set()
    for text in src.values():
        for m in re.finditer(r"launch_dependent\(\s*([A-Za-z_][\w:]*)", text):
            names.add(m.group(1).split("::")[-1])
    return names


def test_every_dependent_launch_names_a_kernel_that_waits():
    src = _sources()
    launched = _launched_kernels(src)
    # the dense launcher passes its chosen instantiation as `kern`
    assert "kern" in launched and "kernel" in launched
    launched -= {"kern", "kernel"}
    launched |= {"dense_tc_kernel", "score_kernel", "score_kernel_staged"}
    assert {"topk_kernel", "topk_slice_kernel", "topk_merge_kernel", "lut_kernel", "dense_f32_kernel",
            "shortlist_csr", "shortlist_ids"} <= launched
    for name in sorted(launched):
        text = next(t for t in src.values() if re.search(r"__global__[^;{]*?\b" + name + r"\s*\(", t, re.S))
        body = _kernel_body(text, name)
        assert "griddep_wait();" in body, f"{name} is launched as a dependent but never waits"
        before = body[:body.index("griddep_wait();")]
        # before the wait: no reads of the kernel's global arguments
        assert "__ldg(" not in before, f"{name} reads global memory before griddep_wait"
        assert not re.search(r"\ba\.(out|offsets|lengths|cand_ids|cand_offsets|pq_codebook|q_scales|t_scales)\b",
                             before), f"{name} touches a global argument before griddep_wait"


def test_plain_launches_are_only_the_standalone_kernels():
    """Kernels still launched with <<<>>> are the E4M3 quantizer and the
    measurement probes.  An ordinary launch starts only after the previous
    kernel has completed, and a dependent launch after it waits for it in
    turn, so mixing the two in one stream keeps the stream's order."""
    plain = set()
    for text in _sources().values():
        for m in re.finditer(r"([A-Za-z_][\w:]*)(?:<[^<>]*>)?<<<", text):
            plain.add(m.group(1).split("::")[-1])
    assert plain <= {"quantize_kernel", "lds_kernel", "read_kernel"}, plain
