"""Source checks of the programmatic dependent launches (no GPU).

A kernel launched with programmatic stream serialisation may start while the
kernel before it on the stream is still running.  It is correct only if it
waits for that grid (griddepcontrol.wait, here pdl_wait / pdl_enter) before it
touches memory the earlier kernels write, and if no path leaves the kernel
before that wait: a grid that could finish before its predecessor would break
the ordering of every kernel after it.  These tests find every kernel the
library launches that way and check both properties in its source.
"""
import pathlib
import re

CSRC = pathlib.Path(__file__).resolve().parents[1] / "paper_1706_00037_gb300" / "csrc"


def _strip_comments(text):
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


SOURCES = {p.name: _strip_comments(p.read_text())
           for p in sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cuh"))}
WAIT = re.compile(r"\bpdl_(wait|enter)\(\)")


def launched_kernels():
    names = set()
    for text in SOURCES.values():
        # call sites, not the helper's own definition
        for m in re.finditer(r"(?<!cudaError_t )launch_pdl\(\s*([A-Za-z_]\w*)", text):
            names.add(m.group(1))
    # the tensor-core products go through cudaLaunchKernelExC with the same attribute
    for text in SOURCES.values():
        if "cudaLaunchAttributeProgrammaticStreamSerialization" in text and \
                "cudaLaunchKernelExC" in text:
            for m in re.finditer(r"cudaLaunchKernelExC\([^;]*?&(\w+)<", text, re.S):
                names.add(m.group(1))
    return names


def kernel_body(name):
    """The body of the __global__ function `name` (text between its braces)."""
    pat = re.compile(r"__global__[^;{]*?\b" + re.escape(name) + r"\s*\(", re.S)
    for text in SOURCES.values():
        m = pat.search(text)
        if not m:
            continue
        depth, i = 1, m.end()
        while depth:  # skip the parameter list
            depth += {"(": 1, ")": -1}.get(text[i], 0)
            i += 1
        start = text.index("{", i)
        depth, j = 1, start + 1
        while depth:
            depth += {"{": 1, "}": -1}.get(text[j], 0)
            j += 1
        return text[start + 1:j - 1]
    raise AssertionError(f"no __global__ definition of {name}")


def test_programmatic_launch_sites_found():
    names = launched_kernels()
    for expected in ("diversify_words", "unpack_bits_bf16", "eval_tc_kernel", "screen_kernel",
                     "ascent_block_kernel", "ascent_warp_kernel", "best_stats_kernel"):
        assert expected in names, expected


def test_every_programmatic_kernel_waits_before_it_can_return():
    for name in sorted(launched_kernels()):
        body = kernel_body(name)
        m = WAIT.search(body)
        assert m, f"{name} never waits for the grid before it"
        before = body[:m.start()]
        assert not re.search(r"\breturn\b", before), f"{name} can return before its wait"


def test_release_only_after_wait():
    """launch_dependents (pdl_release) never precedes the wait in a kernel."""
    for name in sorted(launched_kernels()):
        body = kernel_body(name)
        w = WAIT.search(body)
        r = re.search(r"\bpdl_release\(\)|griddepcontrol\.launch_dependents", body)
        if r:
            assert w and w.start() < r.start(), name


def test_climb_kernels_do_not_release_early():
    """The ascent hands out its first starts by block index and relies on its
    blocks being spread over idle SMs; neither it nor the start-up product in
    front of it lets the next kernel in early."""
    for name in ("ascent_block_kernel", "ascent_warp_kernel"):
        body = kernel_body(name)
        assert "pdl_release" not in body and "pdl_enter" not in body, name
    body = kernel_body("eval_tc_kernel")
    assert re.search(r"if\s*\(\s*!YMODE\s*\)\s*pdl_release\(\)", body)
