"""The Python example of README.md: it compiles (CPU) and runs end to end (GPU)."""
import os
import re

import pytest

from conftest import ROOT


def _example():
    with open(os.path.join(ROOT, "README.md")) as f:
        blocks = re.findall(r"```python\n(.*?)```", f.read(), re.S)
    assert blocks, "README has no Python example"
    return blocks[0]


def test_readme_example_compiles():
    compile(_example(), "README.md", "exec")


@pytest.mark.gpu
@pytest.mark.slow
def test_readme_example_runs(cuda_ok):
    import __graft_entry__
    __graft_entry__.build()
    scope = {}
    exec(compile(_example(), "README.md", "exec"), scope)
    assert abs(scope["r"]["E0"] + 13.6218548212) < 1e-9
    assert scope["status"].shape == scope["E0s"].shape
