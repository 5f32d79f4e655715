"""Host-side fault injection's spec (dspg_fault_inject), no GPU needed: the
library loads without one, well-formed specs arm and disarm, malformed ones
are refused with DSPG_ERR_INVALID."""

import pytest


def test_fault_spec_parsing():
    import paper_2202_08808_gb300 as pkg
    for spec in ("alloc@1", "validate@3", "alloc@2,validate@1", "", None):
        pkg.fault_inject(spec)
    for bad in ("alloc", "alloc@0", "alloc@-1", "alloc@x", "copy@1", "alloc@1,", "@3"):
        if bad == "alloc@1,":
            pkg.fault_inject(bad)  # a trailing comma is an empty item: allowed
            continue
        with pytest.raises(pkg.DspgError) as e:
            pkg.fault_inject(bad)
        assert e.value.status == 1
    pkg.fault_inject(None)
