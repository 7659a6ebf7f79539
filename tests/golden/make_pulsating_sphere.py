"""Writes tests/golden/pulsating_sphere.txt: the surface potential of the unit sphere pulsating with
q = du/dn = 1 as the paper prints it for its radiation benchmark (Sec. 5.2: u = 1/(1 - ik) on the unit
sphere), at the paper's wavenumbers k = 2 pi, 4 pi, 8 pi, 16 pi, 32 pi. The values are the printed
closed form evaluated here in plain complex arithmetic; nothing from oracle/ or the library is used, so
the file can check the oracle's general-radius formula a/(1 - ika)."""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))

if __name__ == "__main__":
    with open(os.path.join(HERE, "pulsating_sphere.txt"), "w") as f:
        f.write("# Sec. 5.2: unit sphere, q = du/dn = 1 (n into the body), u = 1/(1 - i k) on the surface\n")
        f.write("# k  Re(u)  Im(u)\n")
        for m in (1, 2, 4, 8, 16):
            k = 2.0 * math.pi * m
            u = 1.0 / complex(1.0, -k)
            f.write(f"{k:.17g} {u.real:.17g} {u.imag:.17g}\n")
