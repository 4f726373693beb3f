"""The usage example of the README runs as written (GPU)."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu


def test_readme_example_runs():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "README.md")).read()
    block = re.search(r"```python\n(.*?)```", text, re.S).group(1)
    scope = {}
    exec(compile(block, "README.md", "exec"), scope)
    assert scope["tree"].n_nodes > 1 and len(scope["trees"]) == 8
    assert scope["pred"].shape[0] == scope["X"].shape[1]
    assert 32 <= scope["prm"].sort_below <= 2048
