"""Lottery BP(+OSD) syndrome decoder for GB300 (sm_103a)."""
