"""The pins catch the mistakes they are meant to catch.

Each case copies the oracle's source into a temporary directory, plants one
plausible mistake in the copy (a textual replacement), builds it with gcc and
runs a pin against it: the pin must fail.  Only the copy is changed; the
oracle itself is never touched.  CPU only."""
import importlib.util
import os
import shutil

import pytest

import test_oracle_closed_forms as closed
import test_oracle_units as units

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")

MUTANTS = {
    # robust density: the lower of the middle two instead of the upper
    "lower_median": ("  return found[nfound / 2];", "  return found[(nfound - 1) / 2];",
                     lambda o: units.test_octree_robust_median_hand_worked(o, "even")),
    # merge kernel 1 / r^2 instead of 1 / (pi r^2)
    "kernel_without_pi": ("  double kernel = 1.0 / (PI_D * (double)c.r * (double)c.r);",
                          "  double kernel = 1.0 / ((double)c.r * (double)c.r);",
                          closed.test_neb_photons_alone_reproduce_the_longer_paths_of_the_furnace),
    # alias table: a small cell paired with itself instead of a large one
    "alias_paired_with_itself": ("    alias[l] = g;\n", "    alias[l] = l;\n",
                                 lambda o: units.test_alias_selection_frequencies_match_power(
                                     o, [1.0, 2.0, 4.0, 8.0, 100.0])),
    "alias_paired_with_itself_plane": ("    alias[l] = g;\n", "    alias[l] = l;\n",
                                       closed.test_plane_under_two_unequal_sphere_lights),
    # Duff et al. basis: wrong sign of the bitangent's z component
    "bitangent_sign": ("  *b = mk3(bb, sign + n.y * n.y * a, -n.y);", "  *b = mk3(bb, sign + n.y * n.y * a, n.y);",
                       units.test_duff_basis_random_normals),
    # Eq. area: corner parity taken from one coordinate instead of all three
    "area_parity": ("    sum += (uppers & 1) ? -term : term;", "    sum += (uppers & 2) ? -term : term;",
                    units.test_area_matches_polygon_clipping),
    # Sec. 5.2: new cells start at an eighth of the split factor, not a quarter
    "children_eighth": ("    o->fresh_count = (o->split_factor * iter + 3) / 4;",
                        "    o->fresh_count = (o->split_factor * iter + 7) / 8;",
                        units.test_octree_split_hand_worked),
}


def _mutant_oracle(tmp_path, name, old, new):
    src = open(os.path.join(ORACLE_DIR, "neb_oracle.c")).read()
    assert src.count(old) == 1, f"{name}: the text to replace must occur exactly once"
    d = tmp_path / name
    d.mkdir()
    (d / "neb_oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ORACLE_DIR, "neb_oracle.h"), d / "neb_oracle.h")
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}", os.path.join(ORACLE_DIR, "oracle.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    m.HERE = str(d)
    m.SRC = str(d / "neb_oracle.c")
    m.LIB_DIR = str(d / "lib")
    m.LIB = str(d / "lib" / "liboracle.so")
    m._lib = None
    m.build(force=True)
    return m


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_fails_on_planted_mistake(tmp_path, oracle, name):
    old, new, pin = MUTANTS[name]
    pin(oracle)                       # passes on the oracle as it is
    m = _mutant_oracle(tmp_path, name, old, new)
    with pytest.raises(AssertionError):
        pin(m)
