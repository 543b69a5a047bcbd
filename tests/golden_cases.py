"""Reader of the multi-case golden files under tests/golden/: '#' comments,
'case <name>' lines starting a case, then 'key value' lines."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_cases(name):
    cases, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            if k == "case":
                cur = cases.setdefault(v, {})
            else:
                cur[k] = float(v)
    return cases
