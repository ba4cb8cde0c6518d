"""The step-kernel identifiers of the C ABI (include/tn.h) and of the Python binding agree: every
TN_KERNEL_* value of the header has a name in tn.KERNEL_NAMES, and every tensor-core name of the
binding is a value of the header (the SIMT variants 1-7 are documented in the header's comment)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_ids():
    text = open(os.path.join(ROOT, "include", "tn.h")).read()
    enum = re.search(r"enum\s*\{\s*(TN_KERNEL_[^}]*)\}", text).group(1)
    return {name: int(v) for name, v in re.findall(r"(TN_KERNEL_\w+)\s*=\s*(\d+)", enum)}


def test_header_and_binding_kernel_ids_agree():
    from paper_2011_02621_gb300 import tn
    ids = header_ids()
    assert ids["TN_KERNEL_SIMT"] == 0 and ids["TN_KERNEL_SIMT_BOX"] == 8
    for name, v in ids.items():
        assert v in tn.KERNEL_NAMES, name
    values = set(ids.values())
    for v, name in tn.KERNEL_NAMES.items():
        if v >= 8:
            assert v in values, (v, name)
    assert tn.KERNEL_IDS == {n: v for v, n in tn.KERNEL_NAMES.items()}


def test_persistent_forms_named_consistently():
    from paper_2011_02621_gb300 import tn
    for base, stem in ((56, "tcgen05_tma_persist"), (64, "tcgen05_persist_c64"), (72, "tcgen05_persist_loadb"),
                       (80, "tcgen05_persist_c64_loadb")):
        assert [tn.KERNEL_NAMES[base + i] for i in range(3)] == [stem, stem + "_bn128", stem + "_bn64"]
