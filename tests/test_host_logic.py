"""Host-side logic of the Python layer that runs without a GPU: buffer
layout of BatchPlan, the label width of a handle, and argument checks that
fire before any device pointer is used."""
import types

import pytest
import torch

from paper_1011_0093_gb300 import _native as N
from paper_1011_0093_gb300 import batch as B


def test_shared_buffer_parts_are_aligned_and_disjoint():
    sizes = [786432, 1, 255, 256, 257, 0, 3 * 173 * 97]
    offs, total = B._offsets(sizes)
    assert offs[0] == 0 and all(o % B._ALIGN == 0 for o in offs)
    for q in range(len(sizes) - 1):
        assert offs[q] + sizes[q] <= offs[q + 1]            # no overlap
        assert offs[q + 1] - offs[q] < sizes[q] + B._ALIGN  # no more padding than needed
    assert total >= offs[-1] + sizes[-1] and total % B._ALIGN == 0


@pytest.mark.parametrize("max_K,dtype,wide", [(1, torch.uint8, False), (256, torch.uint8, False),
                                              (257, torch.int16, True),
                                              (1024, torch.int16, True)])
def test_label_width_follows_the_palette_limit(max_K, dtype, wide):
    h = types.SimpleNamespace(max_K=max_K)
    assert N.label_dtype(h) == dtype
    assert (int(max_K) > N.MAX_K) == wide
    assert N.MAX_K == 256 and N.MAX_K_WIDE == 1024


def test_label_arrays_of_the_wrong_width_are_refused():
    narrow = torch.zeros(8, dtype=torch.uint8)
    wide = torch.zeros(8, dtype=torch.int16)
    with pytest.raises(ValueError, match="int16"):
        N._lab(narrow, True, "labels", 8)
    with pytest.raises(ValueError, match="uint8"):
        N._lab(wide, False, "labels", 8)
    assert N._lab(None, True, "labels") is None
    # the right width still has to live on the device
    with pytest.raises(ValueError, match="CUDA"):
        N._lab(wide, True, "labels", 8)


def test_pack_places_each_image_at_its_offset_and_checks_shapes():
    shapes = [(3, 5, 3), (2, 2, 4), (7, 1, 3)]
    offs, total = B._offsets(h * w * c for h, w, c in shapes)
    g = torch.Generator().manual_seed(4)
    imgs = [torch.randint(0, 256, s, dtype=torch.uint8, generator=g) for s in shapes]
    buf = torch.full((total,), 77, dtype=torch.uint8)
    B._pack_into(buf, offs, shapes, [im.numpy() for im in imgs])
    for off, im in zip(offs, imgs):
        assert torch.equal(buf[off:off + im.numel()], im.reshape(-1))
    # the padding between parts is left alone
    assert int(buf[offs[0] + imgs[0].numel()]) == 77
    with pytest.raises(ValueError, match="2 images for a plan of 3"):
        B._pack_into(buf, offs, shapes, imgs[:2])
    with pytest.raises(ValueError, match="image 1"):
        B._pack_into(buf, offs, shapes, [imgs[0], imgs[0], imgs[2]])
    with pytest.raises(ValueError, match="uint8"):
        B._pack_into(buf, offs, shapes, [imgs[0], imgs[1].int(), imgs[2]])


def test_tensor_arguments_are_checked_before_any_call():
    cpu = torch.zeros(12, dtype=torch.uint8)
    with pytest.raises(ValueError, match="CUDA"):
        N._dev(cpu, torch.uint8, "rgb")
    assert N._dev(None, torch.uint8, "rgb") is None
    with pytest.raises(ValueError, match="3 or 4 channels"):
        N._pixels(torch.zeros(4, 4, 2, dtype=torch.uint8))
    assert N._pixels(torch.zeros(5, 7, 4, dtype=torch.uint8)) == (35, 4)
    assert N._pixels(torch.zeros(6, 3, dtype=torch.uint8)) == (6, 3)


def test_product_path_never_imports_the_oracle():
    """The package and its sources name no oracle module: importing the
    package (and loading its library) leaves the oracle unloaded."""
    import ast
    import os
    import subprocess
    import sys
    pkg = os.path.dirname(N.__file__)
    for f in sorted(os.listdir(pkg)):
        if f.endswith(".py"):
            tree = ast.parse(open(os.path.join(pkg, f)).read())
            for node in ast.walk(tree):
                names = ([a.name for a in node.names] if isinstance(node, ast.Import) else
                         [node.module or ""] if isinstance(node, ast.ImportFrom) else [])
                assert not any(n.split(".")[0] == "oracle" for n in names), f
    for f in os.listdir(os.path.join(pkg, "csrc")):
        assert "oracle" not in open(os.path.join(pkg, "csrc", f)).read().lower(), f
    from paper_1011_0093_gb300 import build as B
    B.build()
    root = os.path.dirname(pkg)
    code = ("import sys, paper_1011_0093_gb300 as w; w.lib(); "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True,
                         text=True, check=True).stdout.strip()
    assert out == "False"
