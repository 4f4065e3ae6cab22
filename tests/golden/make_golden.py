"""Writes the stored expected values under tests/golden/ that are not transcribed from the paper.

Every value written here comes from the oracle alone (oracle/), never from the CUDA library.
Run: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402


def main():
    with open(os.path.join(HERE, "deal_seed0.txt"), "w") as f:
        f.write(" ".join(str(int(c)) for c in O.deal(0)) + "\n")


if __name__ == "__main__":
    main()
