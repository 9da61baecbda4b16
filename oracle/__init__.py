"""Hopcroft-Tarjan oracle: test infrastructure only (see ht.py)."""
