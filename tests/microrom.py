"""Tiny hand-assembled test cartridges built with the input module's assembler."""
from paper_2606_22447_b300 import synth


def rom4k(build, origin=0xF000, table=True):
    """4K image: `build(asm)` emits code at $F000; an identity table sits at
    $FE00 (value i at $FE00+i) and the reset vector points at $F000."""
    a = synth.Asm(origin, 4096)
    build(a)
    if table:
        a.at(0xE00)
        for i in range(256):
            a.byte(i)
    a.at(4096 - 6)
    a.word(0xF000)
    a.word(0xF000)
    a.word(0xF000)
    return bytes(a.resolve())
