"""Host-side and source checks of the tensor-store epilogue (no GPU needed).

The switch is process-wide and host-only. In the kernel source: the staged block is made
visible to the async proxy (fence.proxy.async) before the tensor store is issued, a
staging block is rewritten only after the previous store from it has finished reading
(wait_group.read), every store has completed (wait_group 0) before the kernel's shared
memory is released, a C load whose wait ran out is drained before that too, and the
host takes the path only for tile rows that are output rows (not for transposed outputs
or the anchor halo) and reads C back in fp32 only."""
import pathlib
import re

from paper_1911_00357_gb300 import binding as B

SRC = (pathlib.Path(__file__).resolve().parents[1] / "paper_1911_00357_gb300" / "csrc" /
       "gemm_tc.cu").read_text()


def test_switch_is_process_wide_and_host_only():
    before = B.ddppo_tma_epilogue()
    try:
        B.ddppo_set_tma_epilogue(False)
        assert B.ddppo_tma_epilogue() is False
        B.ddppo_set_tma_epilogue(True)
        assert B.ddppo_tma_epilogue() is True
    finally:
        B.ddppo_set_tma_epilogue(before)


def _epilogue_path():
    a = SRC.index("if (tma_out) {\n          // tensor-store path")
    b = SRC.index("if (trans_out) {", a)
    return SRC[a:b]


def test_store_ordering_in_the_epilogue():
    p = _epilogue_path()
    # the previous store has read the block before it is rewritten (or loaded into)
    assert p.index("cp.async.bulk.wait_group.read 0") < p.index("tma_load_")
    assert p.index("cp.async.bulk.wait_group.read 0") < p.index("reinterpret_cast<float4*>(sb")
    # the generic-proxy writes are fenced before the tensor store reads them
    fence = p.index("fence.proxy.async.shared::cta")
    assert fence < p.index("tma_store_3d") and fence < p.index("tma_store_2d")
    assert p.index("reinterpret_cast<uint4*>(sb") < fence
    # one commit per issued store
    assert p.count("cp.async.bulk.commit_group") == 1


def test_stores_and_loads_complete_before_the_kernel_ends():
    tail = SRC[SRC.index("if (!ok) break;\n    }\n    // every tensor store"):SRC.index("tcgen05.dealloc")]
    assert "cp.async.bulk.wait_group 0;" in tail
    assert "mbar_drain_wait(&epi_bar[q]" in tail


def test_host_conditions():
    i = SRC.index("int tma_out = 0;")
    cond = SRC[i:SRC.index("::ddppo::launch_k(gemm_tc_kernel<BN>", i)]
    assert "!trans" in cond
    assert re.search(r"ca\.on == 0 \|\| ca\.on == 1 \|\| ca\.on == 4", cond)  # not the anchor halo (3)
    assert "d.beta == 0.f || !d.c_bf16" in cond  # C is read back in fp32 only
    assert "ca.on != 4" in cond  # split-K partials never come from the row halo
