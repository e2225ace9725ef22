"""Host checks of the tensor-core GEMM's descriptor encoders (no GPU needed).

The expected words are composed here by hand from the field tables of the PTX ISA's tcgen05
shared-memory descriptor (start address >> 4 in bits 0-13, leading byte offset >> 4 in bits 16-29,
stride byte offset >> 4 in bits 32-45, bits 46-48 = 0b001, swizzle mode in bits 61-63: 2 = 128-byte
swizzle) and instruction descriptor for kind::f16 (accumulator format F32 = 1 in bits 4-5, A and B
format BF16 = 1 in bits 7-9 and 10-12, K-major = 0 in bits 15 and 16, N / 8 in bits 17-22, M / 16 in
bits 24-28), so a shifted or mis-sized field fails.
"""
import pytest


@pytest.fixture(scope="module")
def lib():
    import paper_2608_09159_gb300 as g
    g.build()
    return g.lib()


def test_smem_descriptor_fields(lib):
    # 1024-byte-aligned tile at 0x400, LBO 16 B, SBO 1024 B, 128-byte swizzle
    want = 0x40 | (1 << 16) | (64 << 32) | (1 << 46) | (2 << 61)
    assert want == 0x4000404000010040
    assert lib.cqp_umma_smem_desc(0x400, 16, 1024, 2) == want
    # the K step inside the atom moves only the start address (32 bytes = 2 units)
    assert lib.cqp_umma_smem_desc(0x400 + 32, 16, 1024, 2) == want + 2
    # the highest shared-memory address keeps 14 bits; larger offsets land in their own fields
    assert lib.cqp_umma_smem_desc(0x3FFF0, 0, 0, 0) == 0x3FFF | (1 << 46)
    assert lib.cqp_umma_smem_desc(0, 0x3FFF0, 0, 0) == (0x3FFF << 16) | (1 << 46)
    assert lib.cqp_umma_smem_desc(0, 0, 0x3FFF0, 0) == (0x3FFF << 32) | (1 << 46)
    # swizzle codes 0 (none), 4 (64 B), 6 (32 B)
    for code in (0, 4, 6):
        assert lib.cqp_umma_smem_desc(0, 0, 0, code) == (1 << 46) | (code << 61)


def test_instruction_descriptor_fields(lib):
    want = (1 << 4) | (1 << 7) | (1 << 10) | ((256 // 8) << 17) | ((128 // 16) << 24)
    assert want == 0x08400490
    assert lib.cqp_umma_instr_desc_bf16(128, 256) == want
    assert lib.cqp_umma_instr_desc_bf16(64, 16) == (1 << 4) | (1 << 7) | (1 << 10) | (2 << 17) | (4 << 24)
    assert lib.cqp_umma_instr_desc_bf16(128, 128) == 0x08200490
