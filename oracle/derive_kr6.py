"""Write oracle/kr6_gamma.txt from the moment conditions in kr6.derive (needs mpmath).

Run:  python oracle/derive_kr6.py
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle import kr6  # noqa: E402


def main():
    vals = kr6.derive()
    lines = ["# Kapur-Rokhlin 6th-order log-correction gamma_j, j = 1..6 (Sec. 2.3),",
             "# derived by oracle/derive_kr6.py from the moment conditions in oracle/kr6.py"]
    for j, v in enumerate(vals, start=1):
        lines.append(f"{j} {float(v):.17e}")
    with open(kr6._TABLE, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
